"""Thin ctypes binding of the C ABI in ``include/sht.h``.

Names follow the C entry points.  This module only marshals arguments:
every step of the transform runs in ``libsht.so`` (host precomputation,
CUDA kernels).  Loading fails loudly if the library has not been built
(``python -m paper_0910_5435_gb300.build``); there is no fallback.

Device buffers are passed as torch CUDA tensors (PyTorch provides device
memory and streams only) or as raw integer addresses.
"""

import ctypes
import os

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libsht.so")

SHT_FP64, SHT_FP32, SHT_SPLIT32, SHT_SPLIT32_ACC64 = 0, 1, 2, 3
PRECISIONS = {"fp64": SHT_FP64, "fp32": SHT_FP32, "split32": SHT_SPLIT32, "split32acc64": SHT_SPLIT32_ACC64}

STATUS = {
    0: "SHT_OK", 1: "SHT_ERR_INVALID_ARG", 2: "SHT_ERR_OOM", 3: "SHT_ERR_CUDA",
    4: "SHT_ERR_PLAN_CORRUPT", 5: "SHT_ERR_TIMEOUT", 6: "SHT_ERR_UNSUPPORTED", 7: "SHT_ERR_NO_DEVICE",
}

# Every symbol declared in include/sht.h.
EXPORTS = [
    "sht_status_string", "sht_plan_opts_default", "sht_plan_create", "sht_plan_create_ex",
    "sht_plan_destroy", "sht_plan_get_stats", "sht_prepare", "sht_plan_nodes", "sht_plan_stream",
    "sht_legendre_synthesize", "sht_legendre_analyze", "sht_legendre_synthesize_adjoint",
    "sht_last_device_status", "sht_direct_prepare", "sht_direct_synthesize", "sht_direct_analyze",
    "sht_workspace_bytes", "sht_phi_synthesize", "sht_phi_analyze", "sht_synthesize", "sht_analyze",
    "sht_last_error_detail", "sht_trace_enable", "sht_trace_read", "sht_legendre_synthesize_noalloc",
    "sht_batch_create", "sht_batch_destroy", "sht_batch_synthesize", "sht_batch_analyze",
    "sht_batch_last_device_status", "sht_batch_autotune", "sht_batch_get_config", "sht_batch_synthesize_adjoint",
    "sht_unit_stats_compute", "sht_gauss_jacobi_nodes", "sht_unit_stats_gauss_jacobi",
    "sht_plan_save", "sht_plan_load", "sht_batch_synthesize_grid", "sht_batch_analyze_grid",
    "sht_measure_fp64_fma", "sht_measure_fp64_mma", "sht_interp_decomp", "sht_plan_stats", "sht_batched_workspace_bytes",
    "sht_synthesize_batched", "sht_analyze_batched", "sht_batch_get_groups",
    "sht_gj_plan_create", "sht_gj_forward", "sht_gj_inverse", "sht_gj_launches",
]

NOALLOC_MAX_SLOTS = 32  # SHT_NOALLOC_MAX_SLOTS


class ShtError(RuntimeError):
    def __init__(self, code, where):
        detail = ""
        if code in (2, 3, 4) and _lib is not None:
            detail = " (" + (_lib.sht_last_error_detail() or b"").decode(errors="replace") + ")"
        super().__init__(f"{where}: {STATUS.get(code, code)}{detail}")
        self.code = code


class sht_plan_opts(ctypes.Structure):
    _fields_ = [
        ("leaf_cols", ctypes.c_int),
        ("trim_eps", ctypes.c_double),
        ("min_band_rows", ctypes.c_int),
        ("host_only", ctypes.c_int),
        ("num_threads", ctypes.c_int),
        ("page_bytes", ctypes.c_int),
        ("eps_fp32", ctypes.c_double),
        ("consumer_warps", ctypes.c_int),
        ("values_inline", ctypes.c_int),
        ("debug_unmet_dependency", ctypes.c_int),
        ("slot_values", ctypes.c_int),
        ("device_build", ctypes.c_int),
        ("device_build_arena_mb", ctypes.c_int),
        ("plan_cache", ctypes.c_char_p),
        ("staging_slots", ctypes.c_int),
    ]


class sht_plan_stats_t(ctypes.Structure):
    _fields_ = [
        ("l", ctypes.c_int),
        ("eps_id", ctypes.c_double),
        ("leaf_cols", ctypes.c_int),
        ("n_units", ctypes.c_int),
        ("n_blocks", ctypes.c_int),
        ("k_max", ctypes.c_int),
        ("k_avg", ctypes.c_double),
        ("k_sigma", ctypes.c_double),
        ("max_abs_T", ctypes.c_double),
        ("max_levels", ctypes.c_int),
        ("n_direct_units", ctypes.c_int),
        ("rows_total", ctypes.c_longlong),
        ("rows_kept", ctypes.c_longlong),
        ("dense_values", ctypes.c_longlong),
        ("factor_values", ctypes.c_longlong),
        ("index_bytes", ctypes.c_longlong),
        ("stream_bytes_fp64", ctypes.c_longlong),
        ("stream_bytes_split32", ctypes.c_longlong),
        ("stream_bytes_fp32", ctypes.c_longlong),
        ("factor_values_fp32", ctypes.c_longlong),
        ("t_quad", ctypes.c_double),
        ("t_comp", ctypes.c_double),
        ("t_upload", ctypes.c_double),
        ("m_max_words", ctypes.c_longlong),
        ("smem_bytes", ctypes.c_int),
        ("page_bytes", ctypes.c_int),
        ("t_factor", ctypes.c_double),
        ("t_factor_kernel", ctypes.c_double),
        ("factor_flops", ctypes.c_double),
        ("id_swaps", ctypes.c_longlong),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None


def lib():
    """The loaded libsht.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_0910_5435_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    vp, c_int, c_double = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.sht_status_string.restype = ctypes.c_char_p
    L.sht_status_string.argtypes = [c_int]
    L.sht_last_error_detail.restype = ctypes.c_char_p
    L.sht_last_error_detail.argtypes = []
    L.sht_plan_opts_default.argtypes = [ctypes.POINTER(sht_plan_opts)]
    L.sht_plan_create.argtypes = [c_int, c_double, ctypes.POINTER(vp)]
    L.sht_plan_create_ex.argtypes = [c_int, c_double, ctypes.POINTER(sht_plan_opts), ctypes.POINTER(vp)]
    L.sht_plan_destroy.argtypes = [vp]
    L.sht_plan_save.argtypes = [vp, ctypes.c_char_p]
    L.sht_plan_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(sht_plan_opts), ctypes.POINTER(vp)]
    L.sht_plan_get_stats.argtypes = [vp, ctypes.POINTER(sht_plan_stats_t)]
    L.sht_prepare.argtypes = [vp, c_int]
    L.sht_plan_nodes.argtypes = [vp, vp, vp]
    L.sht_plan_stream.argtypes = [vp, c_int, c_int, vp, ctypes.POINTER(ctypes.c_size_t),
                                  ctypes.POINTER(ctypes.c_size_t)]
    for name in ["sht_legendre_synthesize", "sht_legendre_analyze", "sht_legendre_synthesize_adjoint"]:
        getattr(L, name).argtypes = [vp, c_int, vp, vp, vp]
    L.sht_last_device_status.argtypes = [vp, vp]
    L.sht_direct_prepare.argtypes = [vp]
    L.sht_direct_synthesize.argtypes = [vp, vp, vp, vp]
    L.sht_direct_analyze.argtypes = [vp, vp, vp, vp]
    L.sht_workspace_bytes.argtypes = [vp, c_int]
    L.sht_workspace_bytes.restype = ctypes.c_size_t
    L.sht_phi_synthesize.argtypes = [vp, c_int, vp, vp, vp, vp]
    L.sht_phi_analyze.argtypes = [vp, c_int, vp, vp, vp]
    L.sht_synthesize.argtypes = [vp, c_int, vp, vp, vp, vp]
    L.sht_analyze.argtypes = [vp, c_int, vp, vp, vp, vp]
    L.sht_trace_enable.argtypes = [vp, c_int]
    L.sht_trace_read.argtypes = [vp, vp, c_int]
    L.sht_legendre_synthesize_noalloc.argtypes = [vp, c_int, vp, vp, c_int, vp, vp]
    L.sht_unit_stats_compute.argtypes = [c_int, c_int, c_int, ctypes.c_double, vp, ctypes.c_ulonglong, vp]
    L.sht_unit_stats_gauss_jacobi.argtypes = [c_int, c_int, c_int, ctypes.c_double, vp, ctypes.c_ulonglong, vp]
    L.sht_gauss_jacobi_nodes.argtypes = [c_int, c_int, c_int, vp, vp]
    L.sht_batch_create.argtypes = [c_int, vp, c_int, vp]
    L.sht_batch_destroy.argtypes = [vp]
    L.sht_batch_synthesize.argtypes = [vp, vp, vp, vp]
    L.sht_batch_analyze.argtypes = [vp, vp, vp, vp]
    L.sht_batch_synthesize_adjoint.argtypes = [vp, vp, vp, vp]
    L.sht_batch_synthesize_grid.argtypes = [vp, vp, vp, vp, vp]
    L.sht_measure_fp64_fma.argtypes = [ctypes.POINTER(c_double)]
    L.sht_measure_fp64_mma.argtypes = [ctypes.POINTER(c_double)]
    L.sht_interp_decomp.argtypes = [vp, c_int, c_int, c_double, ctypes.POINTER(c_int), vp, vp,
                                    ctypes.POINTER(c_int)]
    L.sht_batch_analyze_grid.argtypes = [vp, vp, vp, vp, vp]
    L.sht_batch_last_device_status.argtypes = [vp, vp]
    L.sht_batch_autotune.argtypes = [vp, c_int, vp, vp, c_int, vp]
    L.sht_batch_get_config.argtypes = [vp, c_int, vp, vp, vp, vp]
    L.sht_plan_stats.argtypes = [vp, ctypes.POINTER(sht_plan_stats_t)]
    L.sht_batch_get_groups.argtypes = [vp, c_int, vp, vp]
    L.sht_batched_workspace_bytes.argtypes = [c_int, vp, c_int]
    L.sht_batched_workspace_bytes.restype = ctypes.c_size_t
    L.sht_synthesize_batched.argtypes = [c_int, vp, c_int, vp, vp, vp, vp]
    L.sht_analyze_batched.argtypes = [c_int, vp, c_int, vp, vp, vp, vp]
    L.sht_gj_plan_create.argtypes = [c_int, c_int, c_int, c_double, ctypes.POINTER(sht_plan_opts), ctypes.POINTER(vp)]
    L.sht_gj_forward.argtypes = [vp, c_int, vp, vp, vp]
    L.sht_gj_inverse.argtypes = [vp, c_int, vp, vp, vp]
    L.sht_gj_launches.argtypes = [vp, c_int, c_int, ctypes.POINTER(c_int)]
    for name in EXPORTS:
        if name not in ("sht_status_string", "sht_workspace_bytes", "sht_last_error_detail",
                        "sht_batched_workspace_bytes"):
            getattr(L, name).restype = c_int
    _lib = L
    return L


def _check(code, where):
    if code != 0:
        raise ShtError(code, where)


def _ptr(t):
    """Device address of a torch tensor (or an int address)."""
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def triangle_size(l):
    return (2 * l) * (2 * l + 1) // 2


class Plan:
    """Owns an ``sht_plan_t`` (``sht_plan_create_ex`` / ``sht_plan_destroy``)."""

    def __init__(self, l, eps_id=1e-12, leaf_cols=64, trim_eps=-1.0, min_band_rows=0, host_only=False,
                 num_threads=0, page_bytes=0, eps_fp32=0.0, consumer_warps=0, values_inline=0,
                 debug_unmet_dependency=0, slot_values=0, device_build=False, device_build_arena_mb=0,
                 plan_cache=None, staging_slots=0, _load=None):
        L = lib()
        opts = sht_plan_opts()
        _check(L.sht_plan_opts_default(ctypes.byref(opts)), "sht_plan_opts_default")
        opts.leaf_cols = leaf_cols
        opts.trim_eps = trim_eps
        opts.min_band_rows = min_band_rows
        opts.host_only = 1 if host_only else 0
        opts.num_threads = num_threads
        opts.page_bytes = page_bytes
        opts.eps_fp32 = eps_fp32
        opts.consumer_warps = consumer_warps
        opts.values_inline = values_inline
        opts.debug_unmet_dependency = debug_unmet_dependency
        opts.slot_values = slot_values
        opts.device_build = 1 if device_build else 0
        opts.device_build_arena_mb = device_build_arena_mb
        cache = os.fsencode(plan_cache) if plan_cache is not None else None
        opts.plan_cache = cache
        opts.staging_slots = staging_slots
        h = ctypes.c_void_p()
        if _load is not None:
            _check(L.sht_plan_load(os.fsencode(_load), ctypes.byref(opts), ctypes.byref(h)), "sht_plan_load")
        else:
            _check(L.sht_plan_create_ex(int(l), float(eps_id), ctypes.byref(opts), ctypes.byref(h)),
                   "sht_plan_create_ex")
        self.handle = h
        if _load is not None:
            l = self.stats()["l"]
        self.l = int(l)
        self.host_only = host_only

    @classmethod
    def load(cls, path, **opts):
        """A plan whose factorizations are read from a plan file (sht_plan_load);
        opts are the run-time options (page_bytes, host_only, ...)."""
        return cls(0, _load=path, **opts)

    def save(self, path):
        """Writes the plan's factorizations to a plan file (sht_plan_save)."""
        _check(lib().sht_plan_save(self.handle, os.fsencode(path)), "sht_plan_save")

    def close(self):
        # batches cached on the plan (differentiable batched synthesis) point
        # into its device memory: they go first
        for b in self.__dict__.pop("_autograd_batches", {}).values():
            b.close()
        if getattr(self, "handle", None):
            lib().sht_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def page_bytes(self):
        """Bytes of one record chunk in effect for this plan (plan option page_bytes)."""
        return self.stats()["page_bytes"]

    def stats(self):
        s = sht_plan_stats_t()
        _check(lib().sht_plan_get_stats(self.handle, ctypes.byref(s)), "sht_plan_get_stats")
        return s.as_dict()

    def prepare(self, prec):
        _check(lib().sht_prepare(self.handle, int(prec)), "sht_prepare")

    def nodes(self):
        x = np.zeros(2 * self.l)
        w = np.zeros(2 * self.l)
        _check(lib().sht_plan_nodes(self.handle, x.ctypes.data, w.ctypes.data), "sht_plan_nodes")
        return x, w

    def stream(self, prec, direction):
        """(pages, values): the page region and the value region of a factor stream."""
        n = ctypes.c_size_t(0)
        npg = ctypes.c_size_t(0)
        _check(lib().sht_plan_stream(self.handle, int(prec), int(direction), None, ctypes.byref(n),
                                     ctypes.byref(npg)), "sht_plan_stream")
        buf = np.zeros(n.value, dtype=np.uint8)
        _check(lib().sht_plan_stream(self.handle, int(prec), int(direction), buf.ctypes.data, ctypes.byref(n),
                                     ctypes.byref(npg)), "sht_plan_stream")
        return buf[:npg.value], buf[npg.value:]


class GJPlan(Plan):
    """Owns a single-block plan of the paper's Section 4 matrices
    (``sht_gj_plan_create``): order m, parity 0 (eq. transform) or 1 (eq.
    transform2), size n."""

    def __init__(self, n, m, parity, eps_id=1e-12, leaf_cols=64, host_only=False, page_bytes=0, eps_fp32=0.0,
                 consumer_warps=0, num_threads=0):
        L = lib()
        opts = sht_plan_opts()
        _check(L.sht_plan_opts_default(ctypes.byref(opts)), "sht_plan_opts_default")
        opts.leaf_cols = leaf_cols
        opts.host_only = 1 if host_only else 0
        opts.page_bytes = page_bytes
        opts.eps_fp32 = eps_fp32
        opts.consumer_warps = consumer_warps
        opts.num_threads = num_threads
        h = ctypes.c_void_p()
        _check(L.sht_gj_plan_create(int(n), int(m), int(parity), float(eps_id), ctypes.byref(opts), ctypes.byref(h)),
               "sht_gj_plan_create")
        self.handle = h
        self.l = self.n = int(n)
        self.m, self.parity = int(m), int(parity)
        self.host_only = host_only

    def launches(self, prec, direction):
        c = ctypes.c_int()
        _check(lib().sht_gj_launches(self.handle, int(prec), int(direction), ctypes.byref(c)), "sht_gj_launches")
        return c.value


def sht_gj_forward(plan, prec, beta, alpha, stream=None):
    _check(lib().sht_gj_forward(plan.handle, int(prec), _ptr(beta), _ptr(alpha), _stream(stream)), "sht_gj_forward")


def sht_gj_inverse(plan, prec, alpha, beta, stream=None):
    _check(lib().sht_gj_inverse(plan.handle, int(prec), _ptr(alpha), _ptr(beta), _stream(stream)), "sht_gj_inverse")


def sht_legendre_synthesize(plan, prec, beta, G, stream=None):
    _check(lib().sht_legendre_synthesize(plan.handle, int(prec), _ptr(beta), _ptr(G), _stream(stream)),
           "sht_legendre_synthesize")


def sht_legendre_analyze(plan, prec, G, beta, stream=None):
    _check(lib().sht_legendre_analyze(plan.handle, int(prec), _ptr(G), _ptr(beta), _stream(stream)),
           "sht_legendre_analyze")


def sht_legendre_synthesize_adjoint(plan, prec, G, beta, stream=None):
    _check(lib().sht_legendre_synthesize_adjoint(plan.handle, int(prec), _ptr(G), _ptr(beta), _stream(stream)),
           "sht_legendre_synthesize_adjoint")


def sht_last_device_status(plan, stream=None):
    return lib().sht_last_device_status(plan.handle, _stream(stream))


def sht_direct_prepare(plan):
    _check(lib().sht_direct_prepare(plan.handle), "sht_direct_prepare")


def sht_direct_synthesize(plan, beta, G, stream=None):
    _check(lib().sht_direct_synthesize(plan.handle, _ptr(beta), _ptr(G), _stream(stream)),
           "sht_direct_synthesize")


def sht_direct_analyze(plan, G, beta, stream=None):
    _check(lib().sht_direct_analyze(plan.handle, _ptr(G), _ptr(beta), _stream(stream)), "sht_direct_analyze")


def sht_legendre_synthesize_noalloc(plan, prec, beta, G, slot=0, status=None, stream=None):
    """sht_legendre_synthesize without allocation: the sweep's scratch is a
    static device slot (0 <= slot < NOALLOC_MAX_SLOTS); ``status`` is an
    optional device uint32 receiving the launch status."""
    _check(lib().sht_legendre_synthesize_noalloc(plan.handle, int(prec), _ptr(beta), _ptr(G), int(slot),
                                                 _ptr(status) if status is not None else None,
                                                 _stream(stream)), "sht_legendre_synthesize_noalloc")


class sht_unit_stats(ctypes.Structure):
    _fields_ = [
        ("l", ctypes.c_int), ("m", ctypes.c_int), ("parity", ctypes.c_int), ("n", ctypes.c_int),
        ("rows_kept", ctypes.c_int), ("levels", ctypes.c_int), ("n_blocks", ctypes.c_int), ("k_max", ctypes.c_int),
        ("k_avg", ctypes.c_double), ("k_sigma", ctypes.c_double), ("max_abs_T", ctypes.c_double),
        ("factor_values", ctypes.c_longlong), ("dense_values", ctypes.c_longlong), ("m_max_words", ctypes.c_longlong),
        ("t_quad", ctypes.c_double), ("t_comp", ctypes.c_double), ("eps_fwd", ctypes.c_double),
        ("eps_inv", ctypes.c_double), ("direct", ctypes.c_int),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


def unit_stats(l, m=0, parity=0, eps_id=1e-12, leaf_cols=64, trim_eps=-1.0, min_band_rows=0, seed=1,
               gauss_jacobi=False):
    """Rank statistics, costs and errors of one parity block's butterfly
    (``sht_unit_stats_compute``; host only, any l up to 40000).  With
    gauss_jacobi the block is the paper's n x n matrix at its own nodes, n = l
    (``sht_unit_stats_gauss_jacobi``)."""
    opts = sht_plan_opts()
    _check(lib().sht_plan_opts_default(ctypes.byref(opts)), "sht_plan_opts_default")
    opts.leaf_cols = leaf_cols
    opts.trim_eps = trim_eps
    opts.min_band_rows = min_band_rows
    out = sht_unit_stats()
    fn = lib().sht_unit_stats_gauss_jacobi if gauss_jacobi else lib().sht_unit_stats_compute
    _check(fn(int(l), int(m), int(parity), float(eps_id), ctypes.byref(opts), int(seed), ctypes.byref(out)),
           "sht_unit_stats")
    return out.as_dict()


def gauss_jacobi_nodes(m, parity, n):
    """(x, rho): the paper's nodes and weights (``sht_gauss_jacobi_nodes``)."""
    x = np.zeros(int(n))
    rho = np.zeros(int(n))
    _check(lib().sht_gauss_jacobi_nodes(int(m), int(parity), int(n), x.ctypes.data, rho.ctypes.data),
           "sht_gauss_jacobi_nodes")
    return x, rho


class Batch:
    """Owns an ``sht_batch_t``: many fields, each with its own plan, through
    one launch.  Holds references to its plans (they must outlive it)."""

    def __init__(self, plans, prec):
        self.plans = list(plans)
        self.prec = int(prec)
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle for p in self.plans])
        h = ctypes.c_void_p()
        _check(lib().sht_batch_create(len(self.plans), arr, self.prec, ctypes.byref(h)), "sht_batch_create")
        self.handle = h.value

    def close(self):
        if getattr(self, "handle", None):
            lib().sht_batch_destroy(self.handle)
            self.handle = None

    def launch_handle(self):
        """The handle for a launch.  The batch's field table points into its
        plans' device memory, so a launch after one of them was closed would
        read freed memory: refused here with SHT_ERR_INVALID_ARG."""
        if not self.handle:
            raise ShtError(1, "batch is closed")
        if any(not p.handle for p in self.plans):
            raise ShtError(1, "a plan of this batch was closed")
        return self.handle

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def groups(self, direction):
        """(largest group size class, number of groups) of a direction
        (sht_batch_get_groups): fields sharing a plan are applied together."""
        mx, n = ctypes.c_int(), ctypes.c_int()
        _check(lib().sht_batch_get_groups(self.handle, int(direction), ctypes.byref(mx), ctypes.byref(n)),
               "sht_batch_get_groups")
        return mx.value, n.value

    def config(self, direction):
        v = [ctypes.c_int() for _ in range(4)]
        _check(lib().sht_batch_get_config(self.handle, int(direction), *[ctypes.byref(x) for x in v]),
               "sht_batch_get_config")
        return dict(zip(("consumer_warps", "nstages", "ctas_per_sm", "smem_bytes"), [x.value for x in v]))


def pointer_array(tensors, device="cuda"):
    """Device int64 array of the tensors' addresses (the pointer arrays of
    the batched calls); keep it alive while a launch may read it."""
    import torch
    return torch.tensor([_ptr(t) for t in tensors], dtype=torch.int64, device=device)


def sht_batch_synthesize(batch, beta_ptrs, G_ptrs, stream=None):
    _check(lib().sht_batch_synthesize(batch.launch_handle(), _ptr(beta_ptrs), _ptr(G_ptrs), _stream(stream)),
           "sht_batch_synthesize")


def sht_batch_analyze(batch, G_ptrs, beta_ptrs, stream=None):
    _check(lib().sht_batch_analyze(batch.launch_handle(), _ptr(G_ptrs), _ptr(beta_ptrs), _stream(stream)),
           "sht_batch_analyze")


def sht_batch_synthesize_adjoint(batch, G_ptrs, beta_ptrs, stream=None):
    _check(lib().sht_batch_synthesize_adjoint(batch.launch_handle(), _ptr(G_ptrs), _ptr(beta_ptrs), _stream(stream)),
           "sht_batch_synthesize_adjoint")


def interp_decomp(A, eps):
    """Interpolative decomposition of the real matrix A (sht_interp_decomp):
    returns (skeleton column indices, redundant column indices, T, exchanges)
    with A[:, redundant] ~= A[:, skeleton] @ T."""
    A = np.asfortranarray(np.asarray(A, dtype=np.float64))
    h, w = A.shape
    k = ctypes.c_int()
    sw = ctypes.c_int()
    perm = np.zeros(w, dtype=np.int32)
    T = np.zeros(max(1, (w * w) // 4 + 1), dtype=np.float64)
    _check(lib().sht_interp_decomp(A.ctypes.data, h, w, float(eps), ctypes.byref(k), perm.ctypes.data,
                                   T.ctypes.data, ctypes.byref(sw)), "sht_interp_decomp")
    kk = k.value
    Tm = T[:kk * (w - kk)].reshape(w - kk, kk).T.copy()
    return perm[:kk].copy(), perm[kk:].copy(), Tm, sw.value


def measure_fp64_fma():
    """Float64 FMA throughput of the current device in TFLOP/s
    (sht_measure_fp64_fma)."""
    t = ctypes.c_double()
    _check(lib().sht_measure_fp64_fma(ctypes.byref(t)), "sht_measure_fp64_fma")
    return t.value


def measure_fp64_mma():
    """Float64 tensor-core (8x8x4 warp MMA) throughput of the current device
    in TFLOP/s (sht_measure_fp64_mma)."""
    t = ctypes.c_double()
    _check(lib().sht_measure_fp64_mma(ctypes.byref(t)), "sht_measure_fp64_mma")
    return t.value


def host_pointer_array(tensors):
    """Host array of the tensors' device addresses (the pointer arrays of the
    grid calls, read during the call only)."""
    return (ctypes.c_void_p * len(tensors))(*[_ptr(t) for t in tensors])


def sht_batch_synthesize_grid(batch, betas, values, workspaces, stream=None):
    """Full synthesis of every field (lists of device tensors, one per field)."""
    _check(lib().sht_batch_synthesize_grid(batch.launch_handle(), host_pointer_array(betas), host_pointer_array(values),
                                           host_pointer_array(workspaces), _stream(stream)),
           "sht_batch_synthesize_grid")


def sht_batch_analyze_grid(batch, values, betas, workspaces, stream=None):
    """Full analysis of every field (lists of device tensors, one per field)."""
    _check(lib().sht_batch_analyze_grid(batch.launch_handle(), host_pointer_array(values), host_pointer_array(betas),
                                        host_pointer_array(workspaces), _stream(stream)),
           "sht_batch_analyze_grid")


def sht_batch_last_device_status(batch, stream=None):
    return int(lib().sht_batch_last_device_status(batch.handle, _stream(stream)))


def sht_batch_autotune(batch, direction, in_ptrs, out_ptrs, reps=3, stream=None):
    _check(lib().sht_batch_autotune(batch.launch_handle(), int(direction), _ptr(in_ptrs), _ptr(out_ptrs), int(reps),
                                    _stream(stream)), "sht_batch_autotune")
    return batch.config(direction)


def sht_workspace_bytes(plan, prec):
    return int(lib().sht_workspace_bytes(plan.handle, int(prec)))


def _plan_array(plans):
    return (ctypes.c_void_p * len(plans))(*[p.handle for p in plans])


def sht_plan_stats(plan):
    """The plan statistics (sht_plan_stats, the same call as sht_plan_get_stats)."""
    s = sht_plan_stats_t()
    _check(lib().sht_plan_stats(plan.handle, ctypes.byref(s)), "sht_plan_stats")
    return s.as_dict()


def sht_batched_workspace_bytes(plans, prec):
    return int(lib().sht_batched_workspace_bytes(len(plans), _plan_array(plans), int(prec)))


def sht_synthesize_batched(plans, prec, betas, values, workspace, stream=None):
    """Full synthesis of len(plans) fields in one call (synchronous on stream):
    betas and values are lists of device tensors, workspace one device buffer
    of sht_batched_workspace_bytes(plans, prec) bytes."""
    _check(lib().sht_synthesize_batched(len(plans), _plan_array(plans), int(prec), host_pointer_array(betas),
                                        host_pointer_array(values), _ptr(workspace), _stream(stream)),
           "sht_synthesize_batched")


def sht_analyze_batched(plans, prec, values, betas, workspace, stream=None):
    """Full analysis of len(plans) fields in one call (synchronous on stream)."""
    _check(lib().sht_analyze_batched(len(plans), _plan_array(plans), int(prec), host_pointer_array(values),
                                     host_pointer_array(betas), _ptr(workspace), _stream(stream)),
           "sht_analyze_batched")


def sht_phi_synthesize(plan, prec, G, values, workspace, stream=None):
    _check(lib().sht_phi_synthesize(plan.handle, int(prec), _ptr(G), _ptr(values), _ptr(workspace),
                                    _stream(stream)), "sht_phi_synthesize")


def sht_phi_analyze(plan, prec, values, G, stream=None):
    _check(lib().sht_phi_analyze(plan.handle, int(prec), _ptr(values), _ptr(G), _stream(stream)),
           "sht_phi_analyze")


def sht_synthesize(plan, prec, beta, values, workspace, stream=None):
    _check(lib().sht_synthesize(plan.handle, int(prec), _ptr(beta), _ptr(values), _ptr(workspace),
                                _stream(stream)), "sht_synthesize")


def sht_analyze(plan, prec, values, beta, workspace, stream=None):
    _check(lib().sht_analyze(plan.handle, int(prec), _ptr(values), _ptr(beta), _ptr(workspace),
                             _stream(stream)), "sht_analyze")


TRACE_FIELDS = ("exec_gemv", "exec_control", "wait_dep", "wait_values", "wait_records", "wait_barrier",
                "n_gemv", "n_control", "n_items", "complete")


def sht_trace_enable(plan, enable=True):
    _check(lib().sht_trace_enable(plan.handle, 1 if enable else 0), "sht_trace_enable")


def sht_trace_read(plan, reset=True):
    out = np.zeros(16, dtype=np.uint64)
    _check(lib().sht_trace_read(plan.handle, out.ctypes.data, 1 if reset else 0), "sht_trace_read")
    return {name: int(out[i]) for i, name in enumerate(TRACE_FIELDS)}
