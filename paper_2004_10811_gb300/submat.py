"""Python binding of the C ABI in ``include/submat.h`` (ctypes).

Argument marshalling only: every step of the computation runs in the CUDA
library ``libsubmat.so``.  Torch supplies device memory and the current
stream.  If the library has not been built, importing works but the first
call raises ``SubmatLibraryMissing`` -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsubmat.so")

FP64, FP32, MIXED_BF16_REFINE = 0, 1, 2
_PREC = {"fp64": FP64, "fp32": FP32, "mixed": MIXED_BF16_REFINE, "bf16": MIXED_BF16_REFINE}

STATUS = {
    0: "OK", 1: "INVALID_ARG", 2: "PATTERN", 3: "CUDA", 4: "OOM", 5: "NONFINITE",
    6: "NOT_CONVERGED", 7: "MU_NO_ROOT", 8: "TIMEOUT", 9: "UNSUPPORTED",
}

#: Every entry point declared in include/submat.h.
EXPORTS = (
    "submat_options_default", "submat_plan_create", "submat_plan_destroy", "submat_sign",
    "submat_sign_host", "submat_trace", "submat_mu_search", "submat_sign_backward",
    "submat_plan_value_count", "submat_get_stats", "submat_get_sub_stats", "submat_last_error",
    "submat_debug_tc_gemm", "submat_dense_sign_noalloc", "submat_autotune", "submat_debug_slice_plan",
    "submat_debug_mu_bisect", "submat_debug_fermi_poly", "submat_plan_create_grouped",
)


class SubmatLibraryMissing(RuntimeError):
    pass


class SubmatError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{self.name}: {message}")


class Options(C.Structure):
    _fields_ = [
        ("prec", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int), ("beta_mode", C.c_int),
        ("symmetrize", C.c_int), ("workspace_cap_bytes", C.c_size_t),
        ("refine_rounds", C.c_int), ("timing", C.c_int), ("col_begin", C.c_int), ("col_end", C.c_int),
        ("hp_mode", C.c_int), ("tile_n_ns", C.c_int), ("tile_n_corr", C.c_int), ("tile_n_hp", C.c_int),
        ("iteration", C.c_int), ("adjoint_mode", C.c_int), ("kT", C.c_double),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("nsub", C.c_int32), ("n_min", C.c_int32), ("n_max", C.c_int32), ("waves", C.c_int32),
        ("iters_min", C.c_int32), ("iters_max", C.c_int32), ("not_converged", C.c_int32),
        ("refine_rounds", C.c_int32), ("refine_cg_iters", C.c_int32), ("refine_fallback", C.c_int32),
        ("sum_n2", C.c_double), ("sum_n3", C.c_double),
        ("flops_ns", C.c_double), ("flops_refine", C.c_double), ("max_resid", C.c_double),
        ("ms_gather", C.c_double), ("ms_ns", C.c_double), ("ms_refine", C.c_double),
        ("ms_scatter", C.c_double), ("workspace_bytes", C.c_size_t), ("launches", C.c_int64),
        ("kernel_ms", C.c_double * 8), ("kernel_launches", C.c_int32 * 8), ("kernel_work", C.c_double * 8),
        ("kernel_exec", C.c_double * 8), ("mu_steps", C.c_int32), ("scale_reduced", C.c_int32),
        ("poly_degree", C.c_int32), ("poly_trunc", C.c_double), ("mu_probes", C.c_int32),
        ("dn_dmu", C.c_double),
    ]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if hasattr(v, "__len__") else v
        return out


_lib = None


def load(path: str = LIB_PATH):
    """Load (once) and type the library.  Raises if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise SubmatLibraryMissing(
            f"{path} not found: build it with __graft_entry__.build() (no CPU fallback)")
    lib = C.CDLL(path)
    vp, i32p, i64p, dp = C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_double)
    lib.submat_options_default.argtypes = [C.POINTER(Options)]
    lib.submat_options_default.restype = None
    lib.submat_plan_create.argtypes = [C.c_int, i32p, i64p, i32p, C.POINTER(Options), vp, C.POINTER(vp)]
    lib.submat_plan_create_grouped.argtypes = [C.c_int, i32p, i64p, i32p, i32p, C.POINTER(Options), vp,
                                               C.POINTER(vp)]
    lib.submat_plan_destroy.argtypes = [vp]
    lib.submat_sign.argtypes = [vp, vp, C.c_double, vp, vp]
    lib.submat_sign_host.argtypes = [vp, dp, C.c_double, dp, vp]
    lib.submat_trace.argtypes = [vp, vp, dp, vp]
    lib.submat_mu_search.argtypes = [vp, vp, C.c_double, C.c_double, C.c_double, C.c_int, dp, vp, vp]
    lib.submat_sign_backward.argtypes = [vp, vp, C.c_double, vp, vp, dp, vp]
    lib.submat_autotune.argtypes = [vp, vp, C.c_double, vp, i32p, vp]
    lib.submat_plan_value_count.argtypes = [vp]
    lib.submat_plan_value_count.restype = C.c_int64
    lib.submat_get_stats.argtypes = [vp, C.POINTER(Stats)]
    lib.submat_get_sub_stats.argtypes = [vp, i32p, i32p, dp, dp]
    lib.submat_debug_tc_gemm.argtypes = [C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, C.c_int, C.c_int,
                                         vp, vp, C.c_int, C.c_double, C.c_int, vp]
    lib.submat_dense_sign_noalloc.argtypes = [C.c_int, vp, C.c_double, vp, C.POINTER(C.c_int), vp]
    lib.submat_debug_slice_plan.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, vp, C.c_int,
                                            C.POINTER(C.c_int32)]
    lib.submat_debug_mu_bisect.argtypes = [vp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int,
                                           C.c_double, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_int32),
                                           C.POINTER(C.c_int32), C.POINTER(C.c_double)]
    lib.submat_debug_fermi_poly.argtypes = [C.c_double, C.c_double, C.c_int, vp, C.c_int,
                                            C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_double)]
    lib.submat_last_error.argtypes = []
    lib.submat_last_error.restype = C.c_char_p
    for name in ("submat_plan_create", "submat_plan_create_grouped", "submat_plan_destroy", "submat_sign", "submat_sign_host",
                 "submat_trace", "submat_mu_search", "submat_sign_backward", "submat_get_stats",
                 "submat_get_sub_stats", "submat_debug_tc_gemm", "submat_dense_sign_noalloc",
                 "submat_debug_slice_plan", "submat_debug_mu_bisect", "submat_debug_fermi_poly"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _check(status, allow=()):
    if status == 0 or status in allow:
        return status
    msg = _lib.submat_last_error().decode(errors="replace") if _lib else ""
    raise SubmatError(status, msg)


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _devptr(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


class Plan:
    """A plan for one symmetric block pattern (see ``submat_plan_create``).

    ``prec``: "fp64", "fp32" or "mixed" (BF16 tensor-core Newton-Schulz with
    FP64 refinement).
    """

    def __init__(self, block_sizes, row_ptr, col_idx, prec="fp64", tol=0.0, max_iter=0,
                 beta_mode=0, symmetrize=False, workspace_cap_bytes=0, refine_rounds=0,
                 timing=False, columns=None, hp_mode=0, tile_n_ns=0, tile_n_corr=0, tile_n_hp=0,
                 iteration=0, adjoint_mode=0, kT=0.0, groups=None, stream=None):
        lib = load()
        self._lib = lib
        self.block_sizes = np.ascontiguousarray(block_sizes, dtype=np.int32)
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        opt = Options()
        lib.submat_options_default(C.byref(opt))
        opt.prec = _PREC[prec] if isinstance(prec, str) else int(prec)
        opt.tol = float(tol)
        opt.max_iter = int(max_iter)
        opt.beta_mode = int(beta_mode)
        opt.symmetrize = int(bool(symmetrize))
        opt.workspace_cap_bytes = int(workspace_cap_bytes)
        opt.refine_rounds = int(refine_rounds)
        opt.timing = int(bool(timing))
        opt.hp_mode = int(hp_mode)
        opt.tile_n_ns = int(tile_n_ns)
        opt.tile_n_corr = int(tile_n_corr)
        opt.tile_n_hp = int(tile_n_hp)
        opt.iteration = int(iteration)
        opt.adjoint_mode = int(adjoint_mode)
        opt.kT = float(kT)
        if columns is not None:
            opt.col_begin, opt.col_end = int(columns[0]), int(columns[1])
        self.options = opt
        h = C.c_void_p()
        st = _stream(stream) if stream is not None else C.c_void_p(0)
        if groups is None:
            _check(lib.submat_plan_create(len(self.block_sizes), _ptr(self.block_sizes, C.c_int32),
                                          _ptr(self.row_ptr, C.c_int64), _ptr(self.col_idx, C.c_int32),
                                          C.byref(opt), st, C.byref(h)))
        else:
            self.groups = np.ascontiguousarray(groups, dtype=np.int32)
            _check(lib.submat_plan_create_grouped(len(self.block_sizes), _ptr(self.block_sizes, C.c_int32),
                                                  _ptr(self.row_ptr, C.c_int64), _ptr(self.col_idx, C.c_int32),
                                                  _ptr(self.groups, C.c_int32), C.byref(opt), st, C.byref(h)))
        self._h = h
        self.value_count = int(lib.submat_plan_value_count(h))

    @classmethod
    def from_bsr(cls, m, **kw):
        return cls(m.block_sizes, m.row_ptr, m.col_idx, **kw)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.submat_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- evaluation --------------------------------------------------------
    def sign(self, K, mu, out=None, stream=None, allow_not_converged=False):
        """D = 1/2 (I - sign(K - mu I)) by the submatrix method (device tensors)."""
        import torch
        if out is None:
            out = torch.empty_like(K)
        st = self._lib.submat_sign(self._h, _devptr(K, "K"), float(mu), _devptr(out, "D"), _stream(stream))
        _check(st, allow=(6,) if allow_not_converged else ())
        return out

    def autotune(self, K, mu, out=None, stream=None):
        """Time the tensor-core tile widths on this K (submat_autotune) and keep
        the faster one per phase.  Returns {"ns": w, "correction": w, "sliced": w}
        (zeros for FP64 / FP32 plans); `out` receives D(mu)."""
        import torch
        if out is None:
            out = torch.empty_like(K)
        w = np.zeros(3, dtype=np.int32)
        _check(self._lib.submat_autotune(self._h, _devptr(K, "K"), float(mu), _devptr(out, "D"),
                                         _ptr(w, C.c_int32), _stream(stream)))
        if w[0]:  # mirror the plan's new widths in the Python-side options
            self.options.tile_n_ns, self.options.tile_n_corr, self.options.tile_n_hp = (int(x) for x in w)
        return {"ns": int(w[0]), "correction": int(w[1]), "sliced": int(w[2])}

    def sign_host(self, K, mu, out=None, stream=None):
        """Same with host float64 arrays; host<->device copies happen inside."""
        K = np.ascontiguousarray(K, dtype=np.float64)
        if out is None:
            out = np.empty_like(K)
        _check(self._lib.submat_sign_host(self._h, _ptr(K, C.c_double), float(mu),
                                          _ptr(out, C.c_double), _stream(stream)))
        return out

    def trace(self, D, stream=None):
        tr = C.c_double()
        _check(self._lib.submat_trace(self._h, _devptr(D, "D"), C.byref(tr), _stream(stream)))
        return tr.value

    def mu_search(self, K, n_el, mu0=0.0, tol=1e-9, max_steps=60, out=None, stream=None,
                  allow_no_root=True):
        """Returns (mu, D, status name)."""
        import torch
        if out is None:
            out = torch.empty_like(K)
        mu = C.c_double()
        st = self._lib.submat_mu_search(self._h, _devptr(K, "K"), float(n_el), float(mu0), float(tol),
                                        int(max_steps), C.byref(mu), _devptr(out, "D"), _stream(stream))
        _check(st, allow=(7,) if allow_no_root else ())
        return mu.value, out, STATUS[st]

    def sign_backward(self, K, mu, Dbar, out=None, stream=None, want_dn_dmu=False):
        import torch
        if out is None:
            out = torch.empty_like(K)
        dn = C.c_double()
        _check(self._lib.submat_sign_backward(self._h, _devptr(K, "K"), float(mu), _devptr(Dbar, "Dbar"),
                                              _devptr(out, "Kbar"), C.byref(dn) if want_dn_dmu else None,
                                              _stream(stream)))
        return (out, dn.value) if want_dn_dmu else out

    # -- statistics ----------------------------------------------------------
    def stats(self):
        s = Stats()
        _check(self._lib.submat_get_stats(self._h, C.byref(s)))
        return s.as_dict()

    def sub_stats(self):
        n = len(self.block_sizes)
        dims = np.zeros(n, np.int32)
        iters = np.zeros(n, np.int32)
        resid = np.zeros(n, np.float64)
        beta = np.zeros(n, np.float64)
        _check(self._lib.submat_get_sub_stats(self._h, _ptr(dims, C.c_int32), _ptr(iters, C.c_int32),
                                              _ptr(resid, C.c_double), _ptr(beta, C.c_double)))
        return {"dims": dims, "iters": iters, "resid": resid, "beta": beta}


def make_autograd_sign(plan: Plan):
    """A torch.autograd.Function for K -> D whose backward is the library's
    adjoint (``submat_sign_backward``)."""
    import torch

    class SubmatSign(torch.autograd.Function):
        @staticmethod
        def forward(ctx, K, mu):
            ctx.save_for_backward(K)
            ctx.mu = float(mu)
            return plan.sign(K, float(mu))

        @staticmethod
        def backward(ctx, Dbar):
            (K,) = ctx.saved_tensors
            return plan.sign_backward(K, ctx.mu, Dbar.contiguous()), None

    return SubmatSign.apply


def debug_tc_gemm(A_hi, B_hi, A_lo=None, B_lo=None, n=None, sym=False, res2=None, skip_arrive=False,
                  timeout_s=2.0, stream=None, allow_timeout=False, tile_n=128):
    """Test hook: the grouped tensor-core GEMM alone (include/submat_debug.h).

    A_*, B_*: CUDA bfloat16 or float16 tensors [count, ld, ld], all of one
    dtype; returns (C float32, status name).
    """
    import torch
    lib = load()
    count, ld, ld2 = A_hi.shape
    assert ld == ld2 and A_hi.dtype in (torch.bfloat16, torch.float16) and A_hi.is_contiguous()
    assert all(t is None or t.dtype == A_hi.dtype for t in (B_hi, A_lo, B_lo))
    split = (A_lo is not None) | (2 if A_hi.dtype == torch.float16 else 0)
    C_ = torch.empty((count, ld, ld), dtype=torch.float32, device=A_hi.device)
    ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)
    st = lib.submat_debug_tc_gemm(count, ld, ld if n is None else int(n), ptr(A_hi), ptr(A_lo),
                                  ptr(B_hi), ptr(B_lo), int(split), int(bool(sym)), ptr(C_), ptr(res2),
                                  int(bool(skip_arrive)), float(timeout_s), int(tile_n), _stream(stream))
    _check(st, allow=(8,) if allow_timeout else ())
    return C_, STATUS[st]


def debug_slice_plan(nx, ny, sym_pairs, per_acc, max_acc=4):
    """Host-only test hook (include/submat_debug.h): the launch plan of an exact
    sliced product as an int32 array of (launch, accumulator, p, q, shift) rows."""
    lib = load()
    n = C.c_int32()
    _check(lib.submat_debug_slice_plan(int(nx), int(ny), int(bool(sym_pairs)), int(per_acc), int(max_acc), None, 0,
                                       C.byref(n)))
    out = np.zeros((max(1, n.value), 5), np.int32)
    _check(lib.submat_debug_slice_plan(int(nx), int(ny), int(bool(sym_pairs)), int(per_acc), int(max_acc),
                                       out.ctypes.data_as(C.c_void_p), n.value, C.byref(n)))
    return out[:n.value]


def debug_mu_bisect(levels, n_el, mu0, tol=1e-9, max_steps=60, bound_scale=1.0, probe_err=0.0,
                    with_probes=False):
    """Host-only test hook (include/submat_debug.h): the mu search's bisection on
    the electron count of the given levels, with the spectral bound scaled by
    ``bound_scale`` and, with ``probe_err`` > 0, probes off by that much.
    Returns (mu, steps, N(mu), status), and the probe count with_probes."""
    lib = load()
    lv = np.ascontiguousarray(levels, dtype=np.float64)
    mu, n = C.c_double(), C.c_double()
    steps, probes = C.c_int32(), C.c_int32()
    st = lib.submat_debug_mu_bisect(lv.ctypes.data_as(C.c_void_p), len(lv), float(n_el), float(mu0),
                                    float(tol), int(max_steps), float(bound_scale), float(probe_err),
                                    C.byref(mu), C.byref(steps), C.byref(probes), C.byref(n))
    _check(st, allow=(6, 7))
    out = (mu.value, steps.value, n.value, STATUS[st])
    return out + (probes.value,) if with_probes else out


NOALLOC_MAX_N = 512


def dense_sign_noalloc(K, mu, out=None, stream=None):
    """D = 1/2 (I - sign(K - mu I)) for one dense n x n CUDA float64 matrix,
    through the entry point that allocates no memory (n <= 512).
    Returns (D, iterations)."""
    import torch
    lib = load()
    n = int(K.shape[0])
    if out is None:
        out = torch.empty_like(K)
    it = C.c_int()
    _check(lib.submat_dense_sign_noalloc(n, _devptr(K, "K"), float(mu), _devptr(out, "D"),
                                         C.byref(it), _stream(stream)))
    return out, it.value


def debug_fermi_poly(c, tol=1e-13, max_degree=8191):
    """Host-only test hook (include/submat_debug.h): the finite-temperature
    polynomial for tanh(c x) on [-1, 1].  Returns (r [blocks, 8], degree,
    truncation bound): p(x) = sum_j (sum_q r[j, q] T_{2q+1}(x)) T_j(T_16(x))."""
    lib = load()
    m, blocks, trunc = C.c_int32(), C.c_int32(), C.c_double()
    _check(lib.submat_debug_fermi_poly(float(c), float(tol), int(max_degree), None, 0, C.byref(m),
                                       C.byref(blocks), C.byref(trunc)))
    r = np.zeros(8 * blocks.value, dtype=np.float64)
    _check(lib.submat_debug_fermi_poly(float(c), float(tol), int(max_degree), r.ctypes.data_as(C.c_void_p),
                                       len(r), C.byref(m), C.byref(blocks), C.byref(trunc)))
    return r.reshape(blocks.value, 8), m.value, trunc.value
