"""Python binding of libmbinv: memory-bounded block recursive inverse on GB300.

Argument marshalling only.  Every step of the recursion runs in the CUDA
kernels of ``libmbinv.so``; PyTorch provides device memory and the stream.
Importing the package does not load the library; the first call does, and
fails loudly when the library has not been built (``build()``) - there is no
CPU fallback.

    import paper_1612_00001_gb300 as mb
    ctx = mb.Context(M, k=8, precision="fp64")     # M: 2-D float64/float32 tensor
    n00 = ctx.block(0, 0)                          # N_00, the (0,0) block of M^-1
    full = ctx.all_blocks()
    g = mb.block(M, 8, 2, 5)                       # differentiable N_25
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmbinv.so")
TEST_LIB_PATH = os.path.join(_HERE, "_build", "libmbinv_test.so")

OK, EINVAL, ENOMEM_CAP, ESINGULAR, ENOTCONV, ETIMEOUT, ECUDA, ENOTSUP = range(8)
PRECISION = {"fp64": 0, "fp32": 1, "mixed": 2, "mixed_bf16": 2, "fp64_tc": 3}
SCHEDULE = {"auto": 0, "levels": 1, "bounded": 2}
VARIANT = {"paper": 0, "principal": 1}
DTYPE_F64, DTYPE_F32 = 0, 1

_lock = threading.Lock()
_lib = None


class MbinvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_size_t), ("precision", ctypes.c_int),
                ("device_cap_bytes", ctypes.c_size_t), ("refine_steps", ctypes.c_int),
                ("bf16_slices", ctypes.c_int), ("cuda_stream", ctypes.c_void_p),
                ("pad_seed", ctypes.c_uint64), ("profile", ctypes.c_int), ("schedule", ctypes.c_int),
                ("out_dtype", ctypes.c_int), ("sing_tol", ctypes.c_double), ("variant", ctypes.c_int),
                ("pivot_cond", ctypes.c_int), ("no_graphs", ctypes.c_int), ("reserved", ctypes.c_int),
                ("tune_cache_path", ctypes.c_void_p)]


class Report(ctypes.Structure):
    _fields_ = [("gemm_flops", ctypes.c_double), ("inv_flops", ctypes.c_double), ("seconds", ctypes.c_double),
                ("rel_residual", ctypes.c_double), ("peak_device_bytes", ctypes.c_size_t),
                ("frames", ctypes.c_size_t), ("inversions", ctypes.c_size_t), ("launches", ctypes.c_size_t),
                ("failed_pivot", ctypes.c_int64), ("gemm_device_seconds", ctypes.c_double),
                ("inv_device_seconds", ctypes.c_double), ("gemm_launches", ctypes.c_size_t),
                ("pack_device_seconds", ctypes.c_double), ("inv_panel_device_seconds", ctypes.c_double),
                ("inv_panel_flops", ctypes.c_double), ("inv_update_flops", ctypes.c_double),
                ("inv_panel_launches", ctypes.c_size_t), ("request_frames", ctypes.c_size_t),
                ("planned_device_bytes", ctypes.c_size_t), ("pack_bytes", ctypes.c_double),
                ("host_in_bytes", ctypes.c_double), ("host_out_bytes", ctypes.c_double),
                ("host_spill_bytes", ctypes.c_size_t), ("graph_replays", ctypes.c_size_t),
                ("max_pivot_cond", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("k", ctypes.c_int64), ("i", ctypes.c_int64), ("j", ctypes.c_int64),
                ("M", ctypes.c_void_p), ("ld", ctypes.c_int64), ("out", ctypes.c_void_p), ("ldo", ctypes.c_int64),
                ("status", ctypes.c_int)]


DONE_CB = ctypes.CFUNCTYPE(None, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p)
BLOCK_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                            ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)


class Rbf(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("n", ctypes.c_int64), ("dim", ctypes.c_int64), ("sigma", ctypes.c_double),
                ("gamma", ctypes.c_double)]

# name -> (restype, argtypes) of every entry point the header declares
SIGNATURES = {
    "mbinv_default_options": (None, [ctypes.POINTER(Options)]),
    "mbinv_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                    ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(Options)]),
    "mbinv_block": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                   ctypes.POINTER(Report)]),
    "mbinv_blocks": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                    ctypes.POINTER(Report)]),
    "mbinv_all_blocks": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, DONE_CB,
                                        ctypes.c_void_p, ctypes.POINTER(Report)]),
    "mbinv_block_row": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.POINTER(Report)]),
    "mbinv_block_col": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.POINTER(Report)]),
    "mbinv_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(Report)]),
    "mbinv_batched_blocks": (ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(Problem), ctypes.c_int,
                                            ctypes.POINTER(Options), ctypes.POINTER(Report)]),
    "mbinv_destroy": (None, [ctypes.c_void_p]),
    "mbinv_reload": (ctypes.c_int, [ctypes.c_void_p]),
    "mbinv_create_from_fn": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int64,
                                            ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.POINTER(Options)]),
    "mbinv_rbf_block": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "mbinv_invert_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                            ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]),
    "mbinv_autotune": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_char_p,
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "mbinv_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mbinv_version": (ctypes.c_char_p, []),
    "mbinv_last_cuda_error": (ctypes.c_char_p, []),
}


def build(force: bool = False) -> str:
    """Compiles libmbinv.so in-tree (nvcc, sm_103a)."""
    from . import build_lib
    return build_lib.build(force=force)


def lib():
    """The loaded library.  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libmbinv is not built ({LIB_PATH} missing); call "
                                   "paper_1612_00001_gb300.build() first - there is no CPU fallback")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


_test_lib = None


def test_lib():
    """The test hooks (libmbinv_test.so, not part of the public header): the
    tests and the bench load them; they call into the product library."""
    global _test_lib
    lib()
    with _lock:
        if _test_lib is None:
            if not os.path.exists(TEST_LIB_PATH):
                raise RuntimeError(f"{TEST_LIB_PATH} missing; call paper_1612_00001_gb300.build() first")
            _test_lib = ctypes.CDLL(TEST_LIB_PATH)
    return _test_lib


def _check(status: int, what: str):
    if status != OK:
        L = lib()
        msg = L.mbinv_status_string(status).decode()
        if status == ECUDA:
            msg += ": " + L.mbinv_last_cuda_error().decode()
        raise MbinvError(status, f"{what}: {msg}")


def _torch():
    import torch
    return torch


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float64:
        return DTYPE_F64
    if t.dtype == torch.float32:
        return DTYPE_F32
    raise TypeError(f"unsupported dtype {t.dtype}: use float64 or float32")


def _ptr(t) -> int:
    return t.data_ptr()


def make_options(precision="fp64", cap: int = 0, refine: int = 0, slices: int = 3, stream=None,
                 pad_seed: int = 0, profile: bool = False, schedule="auto", sing_tol: float = 0.0,
                 out_dtype=None, graphs: bool = True, variant="paper", pivot_cond: bool = False,
                 tune_cache_path=None) -> Options:
    o = Options()
    lib().mbinv_default_options(ctypes.byref(o))
    o.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    o.device_cap_bytes = int(cap)
    o.refine_steps = int(refine)
    o.bf16_slices = int(slices)
    o.cuda_stream = stream
    o.pad_seed = int(pad_seed)
    o.profile = int(bool(profile))
    o.schedule = SCHEDULE[schedule] if isinstance(schedule, str) else int(schedule)
    o.sing_tol = float(sing_tol)
    o.no_graphs = 0 if graphs else 1
    o.variant = VARIANT[variant] if isinstance(variant, str) else int(variant)
    o.pivot_cond = int(bool(pivot_cond))
    if tune_cache_path:
        o._path = ctypes.create_string_buffer(str(tune_cache_path).encode())  # kept alive with the options
        o.tune_cache_path = ctypes.cast(o._path, ctypes.c_void_p)
    o.out_dtype = {None: 0, "float64": 1, "float32": 2}[None if out_dtype is None else str(out_dtype).split(".")[-1]]
    return o


class Context:
    """One matrix M (n x n, row-major) split into k x k blocks.

    M may live on the host or on the GPU; a GPU tensor is borrowed and must
    not change while the context lives."""

    def __init__(self, M, k: int, precision="fp64", cap: int = 0, refine: int = 0, slices: int = 3,
                 pad_seed: int = 0, stream=None, profile: bool = False, schedule="auto", sing_tol: float = 0.0,
                 out_dtype=None, graphs: bool = True, variant="paper", pivot_cond: bool = False,
                 tune_cache_path=None):
        torch = _torch()
        if M.dim() != 2 or M.shape[0] != M.shape[1]:
            raise ValueError("M must be square")
        if M.stride(1) != 1:
            M = M.contiguous()
        self.M = M
        self.n = M.shape[0]
        self.k = int(k)
        self.b = -(-self.n // self.k)
        self.mdtype = M.dtype  # type of M, G and dM
        self.dtype = M.dtype if out_dtype is None else out_dtype  # type of the returned blocks
        self.device = M.device if M.is_cuda else torch.device("cuda", torch.cuda.current_device())
        if stream is None:
            stream = torch.cuda.current_stream(self.device).cuda_stream
        self.stream = stream
        self.opts = make_options(precision, cap, refine, slices, stream, pad_seed, profile, schedule, sing_tol,
                                 out_dtype, graphs, variant, pivot_cond, tune_cache_path)
        h = ctypes.c_void_p()
        _check(lib().mbinv_create(ctypes.byref(h), self.n, self.k, _dtype_code(M), _ptr(M), M.stride(0),
                                  ctypes.byref(self.opts)), "mbinv_create")
        self._h = h
        self.last_report = None

    @classmethod
    def from_rbf(cls, x, k: int, sigma: float, gamma: float, dtype=None, precision="fp64_tc", cap: int = 0,
                 stream=None, out_dtype=None):
        """The LS-SVM matrix A_gamma of the points x (n x dim, float64 on the
        GPU) - order n + 1 - produced block by block on the GPU by the
        library's RBF producer and never stored."""
        torch = _torch()
        self = cls.__new__(cls)
        self._keep = x = x.contiguous().to(torch.float64)
        self.rbf = Rbf(_ptr(x), x.shape[0], x.shape[1], float(sigma), float(gamma))
        self.n = x.shape[0] + 1
        self.k = int(k)
        self.b = -(-self.n // self.k)
        self.mdtype = dtype or torch.float64
        self.dtype = self.mdtype if out_dtype is None else out_dtype
        self.device = x.device
        self.stream = torch.cuda.current_stream(self.device).cuda_stream if stream is None else stream
        self.opts = make_options(precision, cap, 0, 3, self.stream, out_dtype=out_dtype)
        L = lib()
        h = ctypes.c_void_p()
        fn = ctypes.cast(L.mbinv_rbf_block, ctypes.c_void_p)
        _check(L.mbinv_create_from_fn(ctypes.byref(h), self.n, self.k,
                                      DTYPE_F64 if self.mdtype == torch.float64 else DTYPE_F32, fn,
                                      ctypes.cast(ctypes.pointer(self.rbf), ctypes.c_void_p),
                                      ctypes.byref(self.opts)), "mbinv_create_from_fn")
        self._h = h
        self.last_report = None
        return self

    def reload(self, M=None):
        """Re-reads M after its contents changed (the next matrix of a stream
        of one shape).  M: optionally new contents, copied into the tensor
        given at construction first (same shape and dtype)."""
        if M is not None:
            if getattr(self, "M", None) is None:
                raise ValueError("this context produces M; there is nothing to reload")
            self.M.copy_(M)
        _check(lib().mbinv_reload(self._h), "mbinv_reload")

    def extent(self, t: int) -> int:
        return self.n - (self.k - 1) * self.b if t == self.k - 1 else self.b

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().mbinv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _out(self, rows, cols, out, on_host=False):
        torch = _torch()
        if out is None:
            dev = torch.device("cpu") if on_host else self.device
            out = torch.empty((rows, cols), dtype=self.dtype, device=dev, pin_memory=False)
        if out.stride(1) != 1 or out.shape[0] < rows or out.shape[1] < cols or out.dtype != self.dtype:
            raise ValueError("out must be a row-major tensor of M's dtype and of sufficient size")
        return out

    def block(self, i: int, j: int, out=None, on_host: bool = False):
        """N_ij (b_i x b_j)."""
        out = self._out(self.extent(i), self.extent(j), out, on_host)
        rep = Report()
        _check(lib().mbinv_block(self._h, i, j, _ptr(out), out.stride(0), ctypes.byref(rep)), f"mbinv_block({i},{j})")
        self.last_report = rep.as_dict()
        return out

    def blocks(self, ij, outs=None, width: int = 0):
        """Several blocks, each by its own run of the recursion, the runs
        executed together.  ij: list of (i, j).  Returns the list of blocks."""
        if outs is None:
            outs = [self._out(self.extent(i), self.extent(j), None) for i, j in ij]
        n = len(ij)
        arr = (ctypes.c_int64 * (2 * n))(*[x for p in ij for x in p])
        ptrs = (ctypes.c_void_p * n)(*[_ptr(o) for o in outs])
        lds = (ctypes.c_int64 * n)(*[o.stride(0) for o in outs])
        rep = Report()
        _check(lib().mbinv_blocks(self._h, n, arr, ptrs, lds, int(width), ctypes.byref(rep)), "mbinv_blocks")
        self.last_report = rep.as_dict()
        return outs

    def all_blocks(self, out=None, done=None, callback=None, on_host: bool = False):
        out = self._out(self.n, self.n, out, on_host)
        rep = Report()
        dbuf = None
        if done is not None:
            flat = bytes(int(bool(x)) for x in done)
            dbuf = ctypes.create_string_buffer(flat, len(flat))
        cb = DONE_CB(lambda i, j, u: callback(int(i), int(j))) if callback else DONE_CB()
        _check(lib().mbinv_all_blocks(self._h, _ptr(out), out.stride(0), dbuf, cb, None, ctypes.byref(rep)),
               "mbinv_all_blocks")
        self.last_report = rep.as_dict()
        return out

    def block_row(self, i: int, out=None):
        out = self._out(self.extent(i), self.n, out)
        rep = Report()
        _check(lib().mbinv_block_row(self._h, i, _ptr(out), out.stride(0), ctypes.byref(rep)), "mbinv_block_row")
        self.last_report = rep.as_dict()
        return out

    def block_col(self, j: int, out=None):
        out = self._out(self.n, self.extent(j), out)
        rep = Report()
        _check(lib().mbinv_block_col(self._h, j, _ptr(out), out.stride(0), ctypes.byref(rep)), "mbinv_block_col")
        self.last_report = rep.as_dict()
        return out

    def backward(self, i: int, j: int, G, dM=None):
        """dM += -(X_i)^T G (Y_j)^T, the gradient of sum(G * N_ij) w.r.t. M."""
        torch = _torch()
        G = G.to(dtype=self.mdtype).contiguous()
        if dM is None:
            dM = torch.zeros((self.n, self.n), dtype=self.mdtype, device=G.device)
        rep = Report()
        _check(lib().mbinv_backward(self._h, i, j, _ptr(G), G.stride(0), _ptr(dM), dM.stride(0), ctypes.byref(rep)),
               "mbinv_backward")
        self.last_report = rep.as_dict()
        return dM


def autotune(b: int, count: int, precision="fp64_tc", cache_path=None):
    """Tunes the panel clusters of batched inverses of order b (see
    mbinv_autotune); returns (bias, seconds per batch)."""
    bias = ctypes.c_int()
    secs = ctypes.c_double()
    p = PRECISION[precision] if isinstance(precision, str) else int(precision)
    _check(lib().mbinv_autotune(int(b), int(count), p, cache_path.encode() if cache_path else None,
                                ctypes.byref(bias), ctypes.byref(secs)), "mbinv_autotune")
    return bias.value, secs.value


def batched_blocks(problems, precision="fp64", cap: int = 0, stream=None):
    """problems: list of (M, k, i, j) with M square tensors of one dtype.
    Returns (list of N_ij tensors, list of statuses)."""
    torch = _torch()
    if not problems:
        return [], []
    dtype = problems[0][0].dtype
    arr = (Problem * len(problems))()
    outs = []
    for t, (M, k, i, j) in enumerate(problems):
        n = M.shape[0]
        b = -(-n // k)
        bi = n - (k - 1) * b if i == k - 1 else b
        bj = n - (k - 1) * b if j == k - 1 else b
        o = torch.empty((bi, bj), dtype=dtype, device=M.device)
        outs.append(o)
        arr[t] = Problem(n, k, i, j, _ptr(M), M.stride(0), _ptr(o), o.stride(0), -1)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    opts = make_options(precision, cap, stream=stream)
    rep = Report()
    st = lib().mbinv_batched_blocks(len(problems), arr, _dtype_code(problems[0][0]), ctypes.byref(opts),
                                    ctypes.byref(rep))
    return outs, [arr[t].status for t in range(len(problems))], rep.as_dict(), st


class _BlockInverse:
    """torch.autograd.Function wrapper (built lazily so that importing the
    package does not import torch)."""
    fn = None

    @classmethod
    def get(cls):
        if cls.fn is None:
            torch = _torch()

            class BlockInverse(torch.autograd.Function):
                @staticmethod
                def forward(ctx, M, k, i, j, precision, cap, refine, variant):
                    c = Context(M.detach(), k, precision=precision, cap=cap, refine=refine, variant=variant)
                    out = c.block(i, j)
                    ctx.mb = c
                    ctx.ij = (i, j)
                    return out

                @staticmethod
                def backward(ctx, G):
                    c = ctx.mb
                    dM = c.backward(ctx.ij[0], ctx.ij[1], G.contiguous())
                    c.close()
                    return dM, None, None, None, None, None, None, None

            cls.fn = BlockInverse
        return cls.fn


def block(M, k: int, i: int, j: int, precision="fp64", cap: int = 0, refine: int = 0, variant="paper"):
    """Differentiable N_ij of M^-1: the backward pass is the hand-written
    adjoint dM = -(X_i)^T G (Y_j)^T, with X_i and Y_j recomputed block by block
    (refine = 1: the forward block refined, and X_i, Y_j taken from the
    whole approximate inverse after Newton-Schulz steps)."""
    return _BlockInverse.get().apply(M, k, i, j, precision, cap, refine, variant)
