"""Thin ctypes binding of the C ABI in include/vk.h (argument marshalling only).

Every numerical step runs inside libvk.so.  PyTorch supplies device memory (through the allocator
callbacks) and CUDA streams; vectors are passed as device pointers of contiguous FP64 tensors.
The library must have been built (``paper_2409_14222_gb300.build.build()``); importing this module
without it raises instead of falling back to anything else.
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libvk.so")

VK_OK = 0
VK_ERR_ARG = 1
VK_ERR_NO_MEMORY = 2
VK_ERR_SINGULAR = 3
VK_ERR_NONFINITE = 4
VK_ERR_NOT_CONVERGED = 5
VK_ERR_TIMEOUT = 6
VK_ERR_CUDA = 7
VK_ERR_INTERNAL = 8
VK_ERR_CANCELLED = 9
VK_BC_DIRICHLET_ALL = 0
VK_CELL_TRIANGLE, VK_CELL_QUAD, VK_CELL_BDM = 0, 1, 2
VK_SERVE_GROUP, VK_SERVE_STREAMS = 0, 1
VK_ASSEMBLY_MATRIX_FULL, VK_ASSEMBLY_MATRIX_FREE = 0, 1

VK_WEIGHTS_PLAIN = 0
VK_WEIGHTS_MULTIPLICITY = 1
VK_PREC_F64 = 0
VK_PREC_F32 = 1
VK_PREC_F64E = 2
VK_CSR_A, VK_CSR_P, VK_CSR_R = 0, 1, 2
VK_BATCH_NONE, VK_BATCH_BF16, VK_BATCH_FP16 = 0, 1, 2
VK_ENGINE_TCGEN05, VK_ENGINE_MMA_SYNC = 0, 1

STATUS_NAMES = {0: "VK_OK", 1: "VK_ERR_ARG", 2: "VK_ERR_NO_MEMORY", 3: "VK_ERR_SINGULAR",
                4: "VK_ERR_NONFINITE", 5: "VK_ERR_NOT_CONVERGED", 6: "VK_ERR_TIMEOUT", 7: "VK_ERR_CUDA",
                8: "VK_ERR_INTERNAL", 9: "VK_ERR_CANCELLED"}

# exported symbols declared in include/vk.h
SYMBOLS = [
    "vk_default_options", "vk_setup", "vk_destroy", "vk_last_error", "vk_footprint", "vk_device_bytes",
    "vk_level_info", "vk_lambda", "vk_residual", "vk_vanka", "vk_smooth", "vk_restrict", "vk_prolong",
    "vk_coarse_solve", "vk_vcycle", "vk_solve", "vk_solve_host", "vk_csr_dims", "vk_export_csr",
    "vk_export_patches", "vk_export_dirichlet", "vk_hessenberg_eigenvalues", "vk_stats_reset", "vk_stats_read",
    "vk_vanka_noalloc", "vk_solve_batch", "vk_apply_schedule", "vk_ndof", "vk_export_dof_coords", "vk_default_server_config", "vk_server_create", "vk_server_submit", "vk_server_wait",
    "vk_server_get_stats", "vk_server_destroy", "vk_check_problem", "vk_server_cancel", "vk_measure_fma_rate",
    "vk_group_create", "vk_group_add", "vk_group_step", "vk_group_result", "vk_group_launches", "vk_group_destroy",
    "vk_group_add_host", "vk_group_active", "vk_manufactured_rhs", "vk_errors",
]


class VkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class vk_problem(ctypes.Structure):
    _fields_ = [("N_coarse", ctypes.c_int32), ("nlevels", ctypes.c_int32), ("k", ctypes.c_int32),
                ("nu", ctypes.c_double), ("bc", ctypes.c_int32), ("domain", ctypes.c_double * 4),
                ("cell", ctypes.c_int32)]


def make_problem(N_coarse, nlevels, k, nu=1.0, bc=VK_BC_DIRICHLET_ALL, domain=(0.0, 1.0, 0.0, 1.0), cell=0):
    return vk_problem(N_coarse, nlevels, k, nu, bc, (ctypes.c_double * 4)(*domain), cell)


class vk_options(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int32), ("weights", ctypes.c_int32), ("cheb_lo", ctypes.c_double),
                ("cheb_hi", ctypes.c_double), ("eig_steps", ctypes.c_int32), ("eig_seed", ctypes.c_uint64),
                ("lambdas", ctypes.POINTER(ctypes.c_double)), ("factor_prec", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("host_threads", ctypes.c_int32), ("host_only", ctypes.c_int32),
                ("max_iterations", ctypes.c_int32), ("batch_prec", ctypes.c_int32),
                ("batch_max_iterations", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("apply_schedule", ctypes.c_int32), ("batch_engine", ctypes.c_int32),
                ("test_expire_wait", ctypes.c_int32), ("spmv_warps", ctypes.c_int32),
                ("batch_coarse_fp32", ctypes.c_int32), ("test_singular_patch", ctypes.c_int32),
                ("patch_assembly", ctypes.c_int32), ("graph_pdl", ctypes.c_int32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class vk_allocator(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("alloc", ALLOC_FN), ("release", RELEASE_FN)]


class vk_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32), ("res0", ctypes.c_double),
                ("res_est", ctypes.c_double), ("true_res", ctypes.c_double),
                ("history", ctypes.POINTER(ctypes.c_double)), ("solve_ms", ctypes.c_double)]


class vk_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("vcycles", ctypes.c_int64), ("apply_launches", ctypes.c_int64),
                ("apply_ms", ctypes.c_double), ("apply_bytes", ctypes.c_double), ("apply_flops", ctypes.c_double),
                ("batch_apply_bytes", ctypes.c_double), ("batch_apply_flops", ctypes.c_double),
                ("spmv_launches", ctypes.c_int64), ("spmv_ms", ctypes.c_double), ("spmv_bytes", ctypes.c_double),
                ("batch_spmv_bytes", ctypes.c_double), ("setup_factor_ms", ctypes.c_double),
                ("setup_ms", ctypes.c_double), ("graph_pdl", ctypes.c_int32)]


class vk_server_config(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("max_per_key", ctypes.c_int32), ("device", ctypes.c_int32),
                ("memory_budget", ctypes.c_size_t), ("options", vk_options), ("mode", ctypes.c_int32)]


class vk_request(ctypes.Structure):
    _fields_ = [("problem", vk_problem), ("b", ctypes.c_void_p), ("rtol", ctypes.c_double),
                ("maxit", ctypes.c_int32)]


class vk_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("res0", ctypes.c_double), ("true_res", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("setup_ms", ctypes.c_double), ("solve_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]


class vk_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("builds", ctypes.c_int64), ("evictions", ctypes.c_int64), ("resident", ctypes.c_int32),
                ("queued", ctypes.c_int32), ("bytes_used", ctypes.c_size_t), ("memory_budget", ctypes.c_size_t),
                ("group_steps", ctypes.c_int64), ("member_steps", ctypes.c_int64)]


_lib = None


def lib():
    """The loaded libvk.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2409_14222_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, D, I, I64, VP = ctypes.POINTER, ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        H = ctypes.c_void_p
        sig = {
            "vk_default_options": (None, [P(vk_options)]),
            "vk_setup": (I, [P(vk_problem), P(vk_options), P(vk_allocator), VP, P(H)]),
            "vk_destroy": (None, [H]),
            "vk_last_error": (ctypes.c_char_p, []),
            "vk_footprint": (I, [P(vk_problem), P(vk_options), P(ctypes.c_size_t)]),
            "vk_device_bytes": (I, [H, P(ctypes.c_size_t)]),
            "vk_level_info": (I, [H, I, P(ctypes.c_int32), P(ctypes.c_int32), P(I64), P(ctypes.c_int32), P(I64)]),
            "vk_lambda": (I, [H, I, P(D)]),
            "vk_residual": (I, [H, I, VP, VP, VP, VP]),
            "vk_vanka": (I, [H, I, VP, VP, VP]),
            "vk_vanka_noalloc": (I, [H, I, VP, VP, VP]),
            "vk_smooth": (I, [H, I, VP, VP, I, VP]),
            "vk_restrict": (I, [H, I, VP, VP, VP]),
            "vk_prolong": (I, [H, I, VP, VP, VP]),
            "vk_coarse_solve": (I, [H, VP, VP, VP]),
            "vk_vcycle": (I, [H, VP, VP, VP]),
            "vk_solve": (I, [H, VP, VP, D, I, P(vk_solve_info), VP]),
            "vk_solve_host": (I, [H, VP, VP, D, I, P(vk_solve_info), VP]),
            "vk_solve_batch": (I, [H, I, VP, I64, VP, D, I, P(vk_solve_info), VP]),
            "vk_csr_dims": (I, [H, I, I, P(ctypes.c_int32), P(ctypes.c_int32), P(I64)]),
            "vk_export_csr": (I, [H, I, I, VP, VP, VP]),
            "vk_export_patches": (I, [H, I, VP, VP, VP]),
            "vk_export_dirichlet": (I, [H, I, VP]),
            "vk_ndof": (I, [H, I, P(I64), P(I64)]),
            "vk_export_dof_coords": (I, [H, I, VP, VP]),
            "vk_hessenberg_eigenvalues": (I, [I, VP, VP, VP]),
            "vk_stats_reset": (I, [H, I]),
            "vk_default_server_config": (None, [P(vk_server_config)]),
            "vk_server_create": (I, [P(vk_server_config), P(VP)]),
            "vk_server_submit": (I, [VP, P(vk_request), P(ctypes.c_uint64)]),
            "vk_server_wait": (I, [VP, ctypes.c_uint64, VP, P(vk_result), I]),
            "vk_server_get_stats": (I, [VP, P(vk_server_stats)]),
            "vk_server_destroy": (None, [VP]),
            "vk_server_cancel": (I, [VP, ctypes.c_uint64]),
            "vk_check_problem": (I, [P(vk_problem), P(vk_options)]),
            "vk_measure_fma_rate": (I, [I, VP, P(D)]),
            "vk_group_create": (I, [I, P(VP)]),
            "vk_group_add": (I, [VP, H, VP, VP, D, I, VP, P(I)]),
            "vk_group_step": (I, [VP, VP, P(I)]),
            "vk_group_result": (I, [VP, I, VP, P(vk_solve_info)]),
            "vk_group_add_host": (I, [VP, H, VP, D, I, VP, P(I)]),
            "vk_group_active": (I, [VP, I, P(I)]),
            "vk_manufactured_rhs": (I, [H, VP]),
            "vk_errors": (I, [H, VP, VP, VP]),
            "vk_group_launches": (I, [VP, P(I64)]),
            "vk_group_destroy": (None, [VP]),
            "vk_stats_read": (I, [H, P(vk_stats)]),
            "vk_apply_schedule": (I, [H, I, P(ctypes.c_int32), P(ctypes.c_int32), P(ctypes.c_int32),
                                      P(ctypes.c_int32), VP, P(ctypes.c_int32)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(code):
    if code != VK_OK:
        raise VkError(code, lib().vk_last_error().decode())
    return code


def default_options(**kw):
    o = vk_options()
    lib().vk_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(t):
    """Device (or host) pointer of a contiguous FP64 tensor / numpy array."""
    if hasattr(t, "data_ptr"):
        assert t.is_contiguous()
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t.ctypes.data)


class TorchAllocator:
    """vk_allocator backed by PyTorch's CUDA caching allocator (keeps the tensors alive)."""

    def __init__(self, device):
        import torch
        self.device = torch.device(device)
        self.live = {}

        def _alloc(ctx, nbytes, stream):
            try:
                t = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
            except Exception:
                return None
            p = t.data_ptr()
            self.live[p] = t
            return p

        def _release(ctx, ptr, stream):
            self.live.pop(ptr, None)

        self._a = ALLOC_FN(_alloc)
        self._r = RELEASE_FN(_release)
        self.struct = vk_allocator(None, self._a, self._r)

    def bytes(self):
        return sum(t.numel() for t in self.live.values())


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(stream)


class Hierarchy:
    """A set-up multigrid hierarchy (vk_setup).  Methods mirror the C ABI names."""

    def __init__(self, N_coarse, nlevels, k, nu=1.0, options=None, device="cuda", host_only=False,
                 lambdas=None, stream=None, allocator="torch", cell=VK_CELL_TRIANGLE):
        self.problem = make_problem(N_coarse, nlevels, k, nu, cell=cell)
        self.options = options if options is not None else default_options()
        if host_only:
            self.options.host_only = 1
        self._lam = None
        if lambdas is not None:
            self._lam = (ctypes.c_double * nlevels)(*[float(v) for v in lambdas])
            self.options.lambdas = self._lam
        self.alloc = None
        aptr = None
        s = ctypes.c_void_p(0)
        if not host_only:
            s = _stream_handle(stream)
            if allocator == "torch":
                self.alloc = TorchAllocator(device)
                aptr = ctypes.byref(self.alloc.struct)
        h = ctypes.c_void_p()
        check(lib().vk_setup(ctypes.byref(self.problem), ctypes.byref(self.options), aptr, s, ctypes.byref(h)))
        self.handle = h
        self.nlevels = nlevels
        self.k = k

    def close(self):
        if getattr(self, "handle", None):
            lib().vk_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- sizes / exports ------------------------------------------------------------------------
    def level_info(self, level):
        nd, nu_, npch = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        nnz, ns = ctypes.c_int64(), ctypes.c_int64()
        check(lib().vk_level_info(self.handle, level, ctypes.byref(nd), ctypes.byref(nu_), ctypes.byref(nnz),
                                  ctypes.byref(npch), ctypes.byref(ns)))
        return dict(ndof=nd.value, n_u=nu_.value, nnz=nnz.value, npatch=npch.value, nslots=ns.value)

    def ndof(self, level=None):
        return self.level_info(self.nlevels - 1 if level is None else level)["ndof"]

    def device_bytes(self):
        b = ctypes.c_size_t()
        check(lib().vk_device_bytes(self.handle, ctypes.byref(b)))
        return b.value

    def lam(self, level):
        v = ctypes.c_double()
        check(lib().vk_lambda(self.handle, level, ctypes.byref(v)))
        return v.value

    def export_csr(self, level, which=VK_CSR_A):
        import numpy as np
        nr, nc, nnz = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        check(lib().vk_csr_dims(self.handle, level, which, ctypes.byref(nr), ctypes.byref(nc), ctypes.byref(nnz)))
        ptr = np.zeros(nr.value + 1, np.int32)
        col = np.zeros(nnz.value, np.int32)
        val = np.zeros(nnz.value, np.float64)
        check(lib().vk_export_csr(self.handle, level, which, _ptr(ptr), _ptr(col), _ptr(val)))
        return (nr.value, nc.value), ptr, col, val

    def export_patches(self, level):
        import numpy as np
        info = self.level_info(level)
        ptr = np.zeros(info["npatch"] + 1, np.int32)
        dofs = np.zeros(info["nslots"], np.int32)
        kind = np.zeros(info["npatch"], np.int8)
        check(lib().vk_export_patches(self.handle, level, _ptr(ptr), _ptr(dofs), _ptr(kind)))
        return ptr, dofs, kind

    def dof_counts(self, level=None):
        """(n_u, n_p) of a level (vk_ndof)."""
        nu_, np_ = ctypes.c_int64(), ctypes.c_int64()
        check(lib().vk_ndof(self.handle, self.nlevels - 1 if level is None else level, ctypes.byref(nu_),
                            ctypes.byref(np_)))
        return nu_.value, np_.value

    def export_dof_coords(self, level):
        """(xy[ndof, 2], kind[ndof]) of a level: node coordinates, 0/1 velocity component, 2 pressure."""
        import numpy as np
        n = self.ndof(level)
        xy = np.zeros((n, 2), np.float64)
        kind = np.zeros(n, np.int8)
        check(lib().vk_export_dof_coords(self.handle, level, _ptr(xy), _ptr(kind)))
        return xy, kind

    def export_dirichlet(self, level):
        import numpy as np
        out = np.zeros(self.ndof(level), np.uint8)
        check(lib().vk_export_dirichlet(self.handle, level, _ptr(out)))
        return out.astype(bool)

    def apply_schedule(self, level):
        """Launch shape of the patch application on a level and the autotuner's candidate times."""
        import numpy as np
        v = [ctypes.c_int32() for _ in range(5)]
        us = np.zeros(16)
        check(lib().vk_apply_schedule(self.handle, level, ctypes.byref(v[0]), ctypes.byref(v[1]),
                                      ctypes.byref(v[2]), ctypes.byref(v[3]), _ptr(us), ctypes.byref(v[4])))
        return dict(split=v[0].value, threads=v[1].value, per_sm=v[2].value, index=v[3].value,
                    cand_us=us[:v[4].value].tolist())

    def stats_reset(self, time_kernels=False):
        check(lib().vk_stats_reset(self.handle, int(time_kernels)))

    def stats(self):
        st = vk_stats()
        check(lib().vk_stats_read(self.handle, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in vk_stats._fields_}

    def manufactured_rhs(self):
        """Right-hand side of the manufactured problem (Eq. model_problem) on the finest level (numpy)."""
        import numpy as np
        b = np.zeros(self.ndof())
        check(lib().vk_manufactured_rhs(self.handle, _ptr(b)))
        return b

    def errors(self, x, stream=None):
        """(relative H^1 velocity, relative L^2 velocity, L^2 pressure) errors of x (vk_errors)."""
        import numpy as np
        e = np.zeros(3)
        check(lib().vk_errors(self.handle, _ptr(x), _ptr(e), _stream_handle(stream)))
        return tuple(float(v) for v in e)

    # ---- device operations (tensors: contiguous float64 on the device) ---------------------------
    def residual(self, level, b, x, r, stream=None):
        check(lib().vk_residual(self.handle, level, _ptr(b), _ptr(x), _ptr(r), _stream_handle(stream)))

    def vanka(self, level, r, z, stream=None):
        check(lib().vk_vanka(self.handle, level, _ptr(r), _ptr(z), _stream_handle(stream)))

    def vanka_noalloc(self, level, r, z, stream=None):
        """vk_vanka without any device allocation (corrections in the library's fixed device array)."""
        check(lib().vk_vanka_noalloc(self.handle, level, _ptr(r), _ptr(z), _stream_handle(stream)))

    def smooth(self, level, b, x, zero_init, stream=None):
        check(lib().vk_smooth(self.handle, level, _ptr(b), _ptr(x), int(zero_init), _stream_handle(stream)))

    def restrict(self, fine_level, r_fine, r_coarse, stream=None):
        check(lib().vk_restrict(self.handle, fine_level, _ptr(r_fine), _ptr(r_coarse), _stream_handle(stream)))

    def prolong(self, fine_level, e_coarse, x_fine, stream=None):
        check(lib().vk_prolong(self.handle, fine_level, _ptr(e_coarse), _ptr(x_fine), _stream_handle(stream)))

    def coarse_solve(self, b, x, stream=None):
        check(lib().vk_coarse_solve(self.handle, _ptr(b), _ptr(x), _stream_handle(stream)))

    def vcycle(self, b, x, stream=None):
        check(lib().vk_vcycle(self.handle, _ptr(b), _ptr(x), _stream_handle(stream)))

    def _info(self, maxit, want_history):
        import numpy as np
        info = vk_solve_info()
        hist = None
        if want_history:
            hist = np.zeros(maxit + 1)
            info.history = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        return info, hist

    def solve(self, b, x, rtol=1e-8, maxit=100, stream=None, history=True, raise_on_nonconv=False):
        """FGMRES solve (vk_solve).  Returns a dict with iterations, converged, history, ..."""
        info, hist = self._info(maxit, history)
        code = lib().vk_solve(self.handle, _ptr(b), _ptr(x), float(rtol), int(maxit), ctypes.byref(info),
                              _stream_handle(stream))
        if code != VK_OK and not (code == VK_ERR_NOT_CONVERGED and not raise_on_nonconv):
            check(code)
        return self._result(info, hist, code)

    def solve_batch(self, B, X, rtol=1e-8, maxit=60, stream=None):
        """vk_solve_batch on column-major device blocks: B, X are (nrhs, ndof) contiguous tensors
        (row r = right-hand side r, i.e. column-major ndof x nrhs).  Returns a list of per-column dicts."""
        nrhs, n = B.shape
        infos = (vk_solve_info * nrhs)()
        code = lib().vk_solve_batch(self.handle, nrhs, _ptr(B), n, _ptr(X), float(rtol), int(maxit), infos,
                                    _stream_handle(stream))
        if code not in (VK_OK, VK_ERR_NOT_CONVERGED):
            check(code)
        return [self._result(infos[r], None, code) for r in range(nrhs)]

    def solve_host(self, b_host, x_host, rtol=1e-8, maxit=100, stream=None, history=False):
        info, hist = self._info(maxit, history)
        code = lib().vk_solve_host(self.handle, _ptr(b_host), _ptr(x_host), float(rtol), int(maxit),
                                   ctypes.byref(info), _stream_handle(stream))
        if code not in (VK_OK, VK_ERR_NOT_CONVERGED):
            check(code)
        return self._result(info, hist, code)

    @staticmethod
    def _result(info, hist, code):
        out = dict(iterations=info.iterations, converged=bool(info.converged), res0=info.res0,
                   res_est=info.res_est, true_res=info.true_res, solve_ms=info.solve_ms, status=code)
        if hist is not None:
            out["history"] = hist[:info.iterations + 1].copy()
        return out


class Group:
    """Several independent solves advanced together, one launch per stage over all members (vk_group_*)."""

    def __init__(self, max_members=8):
        self.handle = ctypes.c_void_p()
        check(lib().vk_group_create(int(max_members), ctypes.byref(self.handle)))
        self._keep = {}

    def add(self, hier, b, x, rtol=1e-8, maxit=100, stream=None):
        """Adds a solve of hier's finest system (b, x: contiguous FP64 device tensors); returns its member id."""
        m = ctypes.c_int()
        check(lib().vk_group_add(self.handle, hier.handle, _ptr(b), _ptr(x), float(rtol), int(maxit),
                                 _stream_handle(stream), ctypes.byref(m)))
        self._keep[m.value] = (hier, b, x, maxit)
        return m.value

    def step(self, stream=None):
        """One FGMRES iteration of every active member; returns the number still active."""
        a = ctypes.c_int()
        check(lib().vk_group_step(self.handle, _stream_handle(stream), ctypes.byref(a)))
        return a.value

    def run(self, stream=None):
        while self.step(stream) > 0:
            pass

    def result(self, member):
        import numpy as np
        maxit = self._keep[member][3]
        info = vk_solve_info()
        hist = np.zeros(maxit + 1)
        info.history = hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        code = lib().vk_group_result(self.handle, int(member), None, ctypes.byref(info))
        if code not in (VK_OK, VK_ERR_NOT_CONVERGED):
            check(code)
        del self._keep[member]
        return Hierarchy._result(info, hist, code)

    def launches(self):
        v = ctypes.c_int64()
        check(lib().vk_group_launches(self.handle, ctypes.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "handle", None):
            lib().vk_group_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def footprint(N_coarse, nlevels, k, nu=1.0, options=None, cell=VK_CELL_TRIANGLE):
    p = make_problem(N_coarse, nlevels, k, nu, cell=cell)
    o = options if options is not None else default_options()
    b = ctypes.c_size_t()
    check(lib().vk_footprint(ctypes.byref(p), ctypes.byref(o), ctypes.byref(b)))
    return b.value


def hessenberg_eigenvalues(H):
    import numpy as np
    H = np.ascontiguousarray(H, dtype=np.float64)
    m = H.shape[0]
    re, im = np.zeros(m), np.zeros(m)
    check(lib().vk_hessenberg_eigenvalues(m, _ptr(H), _ptr(re), _ptr(im)))
    return re + 1j * im


def measure_fma_rate(fp64=True, stream=None):
    """FMA throughput of the current device in TFLOP/s (vk_measure_fma_rate), FP64 or FP32."""
    v = ctypes.c_double()
    check(lib().vk_measure_fma_rate(0 if fp64 else 1, _stream_handle(stream), ctypes.byref(v)))
    return v.value


def ndof_of(N_coarse, nlevels, k):
    """DoFs of the finest level (canonical numbering of include/vk.h)."""
    Nf = N_coarse << (nlevels - 1)
    return 2 * (k * Nf + 1) ** 2 + ((k - 1) * Nf + 1) ** 2


class Server:
    """The solve service of include/vk.h (vk_server_*): submit host right-hand sides, wait for results."""

    def __init__(self, slots=4, memory_budget=0, device=0, options=None, max_per_key=None, mode=VK_SERVE_GROUP):
        c = vk_server_config()
        lib().vk_default_server_config(ctypes.byref(c))
        c.slots = slots
        c.mode = mode
        if max_per_key is not None:
            c.max_per_key = max_per_key
        c.memory_budget = int(memory_budget)
        c.device = device
        if options is not None:
            c.options = options
        self.handle = ctypes.c_void_p()
        check(lib().vk_server_create(ctypes.byref(c), ctypes.byref(self.handle)))
        self._keep = {}

    def submit(self, N_coarse, nlevels, k, b, rtol=1e-8, maxit=100, nu=1.0):
        import numpy as np
        b = np.ascontiguousarray(b, dtype=np.float64)
        assert b.size == ndof_of(N_coarse, nlevels, k)
        r = vk_request(make_problem(N_coarse, nlevels, k, nu), b.ctypes.data, float(rtol), int(maxit))
        t = ctypes.c_uint64()
        check(lib().vk_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t)))
        self._keep[t.value] = ndof_of(N_coarse, nlevels, k)
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        """Returns (x, result dict); raises VkError(VK_ERR_TIMEOUT) if not ready in time."""
        import numpy as np
        n = self._keep[ticket]
        x = np.zeros(n)
        res = vk_result()
        check(lib().vk_server_wait(self.handle, ctypes.c_uint64(ticket), x.ctypes.data_as(ctypes.c_void_p),
                                   ctypes.byref(res), int(timeout_ms)))
        del self._keep[ticket]
        return x, {name: getattr(res, name) for name, _ in vk_result._fields_}

    def cancel(self, ticket):
        """vk_server_cancel: drop a request that is still queued (its wait then reports VK_ERR_CANCELLED)."""
        check(lib().vk_server_cancel(self.handle, ctypes.c_uint64(ticket)))

    def stats(self):
        st = vk_server_stats()
        check(lib().vk_server_get_stats(self.handle, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in vk_server_stats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib().vk_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
