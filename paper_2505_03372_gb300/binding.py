"""Thin ctypes binding of libwt (include/wt.h).

Argument marshalling only: every step of construction and every query runs in
libwt's CUDA kernels.  PyTorch supplies device memory and the current stream.
If libwt.so is missing or cannot be loaded this module raises at import of the
first call; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# WT_LIB_VARIANT=debug loads libwt_debug.so: the same library with every load of
# a query walk bounds-checked (a failed check reports WT_EBOUNDS)
LIB_PATH = os.path.join(_HERE, "libwt_debug.so" if os.environ.get("WT_LIB_VARIANT") == "debug" else "libwt.so")

WT_OK, WT_EINVAL, WT_ESYMBOL, WT_ENOMEM, WT_ECUDA, WT_EQUERY, WT_ETIMEOUT, WT_EUNSUPPORTED, WT_EBOUNDS = range(9)
EXPORT_BITS, EXPORT_L1, EXPORT_L2, EXPORT_S0, EXPORT_S1, EXPORT_C, EXPORT_CODES, EXPORT_LENS, EXPORT_NODES = range(9)
EXPORT_EPS0, EXPORT_EPS1, EXPORT_MLP, EXPORT_RESID0, EXPORT_RESID1 = 9, 10, 11, 12, 13
ANCHOR = 4  # select samples per anchor segment of the learned select
LEARN_NONE, LEARN_PLA, LEARN_MLP = 0, 1, 2
MLP_PARAMS = 97
MAX_LEVELS = 26

# every symbol include/wt.h declares (checked by the ABI test)
EXPORTED = (
    "wt_build", "wt_build_host", "wt_destroy", "wt_access", "wt_rank", "wt_select", "wt_query_mixed", "wt_query_host", "wt_status_sync",
    "wt_info", "wt_export", "wt_status_str", "wt_profile_enable", "wt_profile_reset", "wt_profile_launches",
    "wt_profile_report", "wt_bitvector_support_static", "wt_train_select", "wt_select_learned", "wt_learned_info",
    "wt_mlp_gradient", "wt_batch_create", "wt_batch_set_queries", "wt_batch_run", "wt_batch_status_sync",
    "wt_batch_tree", "wt_batch_bytes", "wt_batch_destroy", "wt_selftest_lookback_timeout", "wt_bitvector_rank",
    "wt_bitvector_select", "wt_alphabet", "wt_order_queries", "wt_walk_ordered", "wt_order_destroy",
)

# wt_order_queries kinds
ORDER_ACCESS, ORDER_RANK, ORDER_SELECT, ORDER_MIXED = 0, 1, 2, 3


class Order:
    """A query batch sorted by walk key (wt_order_queries); see Tree.order,
    Tree.walk.  close(stream) releases it after the work queued on `stream`."""

    def __init__(self, tree, kind, arg, c=None, kinds=None, stream=None):
        import torch

        if kind not in (ORDER_ACCESS, ORDER_RANK, ORDER_SELECT, ORDER_MIXED):
            raise ValueError("kind must be one of ORDER_ACCESS, ORDER_RANK, ORDER_SELECT, ORDER_MIXED")
        self.kind, self.q, self.device = kind, arg.numel(), arg.device
        if kind != ORDER_ACCESS and (c is None or c.numel() != self.q):
            raise ValueError("c must have arg's length")
        if kind == ORDER_MIXED and (kinds is None or kinds.numel() != self.q or kinds.dtype != torch.uint8):
            raise ValueError("kinds must be uint8 with arg's length")
        self._stream = stream
        h = ctypes.c_void_p()
        dk = _dptr(kinds, "kinds") if kind == ORDER_MIXED and self.q else None
        dc = _as_u32(c, "c") if kind != ORDER_ACCESS and self.q else None
        da = _as_u64(arg, "arg") if self.q else None
        _check(lib().wt_order_queries(tree._h, kind, dk, dc, da, self.q, _stream(stream), ctypes.byref(h)),
               "wt_order_queries")
        self._h = h.value

    def close(self, stream=None):
        if self._h:
            h, self._h = self._h, None
            _check(lib().wt_order_destroy(h, _stream(stream)), "wt_order_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class WTError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_str(status)}" if what else status_str(status))


LAYOUT_TREE, LAYOUT_MATRIX = 0, 1


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    """wt_allocator: alloc(bytes, stream, ctx) / free(ptr, stream, ctx) callbacks."""
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [("sample_k", ctypes.c_uint32), ("layout", ctypes.c_uint32),
                ("allocator", ctypes.POINTER(Allocator)), ("reserved", ctypes.c_uint32 * 4)]


class TorchAllocator:
    """A wt_allocator backed by PyTorch's CUDA caching allocator, so trees and
    scratch buffers live in torch's memory pool.  libwt asks for memory on the
    caller's stream and returns it on the same stream, which is how the
    caching allocator orders reuse.  A failed allocation returns NULL (libwt
    then reports WT_ENOMEM).  Keep the object alive as long as any tree built
    with it."""

    def __init__(self, device=None):
        import torch

        self.device = torch.cuda.current_device() if device is None else int(device)

        def _alloc(nbytes, stream, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), self.device, int(stream or 0))
            except Exception:
                return None

        def _free(ptr, stream, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        self._fa, self._ff = _ALLOC_FN(_alloc), _FREE_FN(_free)
        self.struct = Allocator(self._fa, self._ff, None)


_torch_allocators = {}


def torch_allocator(device=None) -> TorchAllocator:
    """The shared TorchAllocator of a device (created on first use)."""
    import torch

    d = torch.cuda.current_device() if device is None else int(device)
    if d not in _torch_allocators:
        _torch_allocators[d] = TorchAllocator(d)
    return _torch_allocators[d]


class Info(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint64),
        ("sigma", ctypes.c_uint32),
        ("levels", ctypes.c_uint32),
        ("symbol_bytes", ctypes.c_uint32),
        ("sample_k", ctypes.c_uint32),
        ("level_size", ctypes.c_uint64 * MAX_LEVELS),
        ("level_ones", ctypes.c_uint64 * MAX_LEVELS),
        ("tree_bytes", ctypes.c_uint64),
        ("layout", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
    ]


class TrainOptions(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint32), ("pairs", ctypes.c_uint32), ("lr", ctypes.c_float),
                ("reserved", ctypes.c_uint32 * 5)]


class LearnedInfo(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_uint32),
        ("pad", ctypes.c_uint32),
        ("fallbacks", ctypes.c_uint64),
        ("model_bytes", ctypes.c_uint64),
        ("eps_mean", (ctypes.c_double * 2) * MAX_LEVELS),
        ("eps_max", (ctypes.c_uint32 * 2) * MAX_LEVELS),
        ("anchor_bytes", ctypes.c_uint64),
    ]


class BatchOptions(ctypes.Structure):
    _fields_ = [("sample_k", ctypes.c_uint32), ("query_threads", ctypes.c_uint32),
                ("allocator", ctypes.POINTER(Allocator)), ("lp_ctas_per_sm", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 3)]


_lib = None


def lib():
    """Load libwt.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libwt.so not found at {LIB_PATH}: run __graft_entry__.build() first")
        L = ctypes.CDLL(LIB_PATH)
        vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
        L.wt_build.argtypes = [vp, u64, u32, u32, ctypes.POINTER(Options), vp, ctypes.POINTER(vp)]
        L.wt_build_host.argtypes = [vp, u64, u32, u32, ctypes.POINTER(Options), vp, ctypes.POINTER(vp)]
        L.wt_destroy.argtypes = [vp]
        L.wt_destroy.restype = None
        L.wt_access.argtypes = [vp, vp, vp, u64, vp]
        L.wt_rank.argtypes = [vp, vp, vp, vp, u64, vp]
        L.wt_select.argtypes = [vp, vp, vp, vp, u64, vp]
        L.wt_query_mixed.argtypes = [vp, vp, vp, vp, vp, u64, vp]
        L.wt_order_queries.argtypes = [vp, u32, vp, vp, vp, u64, vp, ctypes.POINTER(vp)]
        L.wt_walk_ordered.argtypes = [vp, vp, vp, vp]
        L.wt_order_destroy.argtypes = [vp, vp]
        L.wt_query_host.argtypes = [vp, u32, vp, vp, vp, vp, u64, u64, vp]
        L.wt_status_sync.argtypes = [vp, vp]
        L.wt_info.argtypes = [vp, ctypes.POINTER(Info)]
        L.wt_export.argtypes = [vp, u32, u32, vp, ctypes.POINTER(u64)]
        L.wt_status_str.argtypes = [ctypes.c_int]
        L.wt_status_str.restype = ctypes.c_char_p
        L.wt_profile_enable.argtypes = [ctypes.c_int]
        L.wt_profile_enable.restype = None
        L.wt_profile_reset.argtypes = []
        L.wt_profile_reset.restype = None
        L.wt_profile_launches.argtypes = []
        L.wt_profile_launches.restype = u64
        L.wt_profile_report.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
        L.wt_profile_report.restype = ctypes.c_size_t
        L.wt_bitvector_support_static.argtypes = [vp, u64, u32, vp, vp, vp, vp, u64, vp, vp, vp]
        L.wt_bitvector_support_static.restype = ctypes.c_int
        L.wt_bitvector_rank.argtypes = [vp, u64, vp, vp, vp, vp, u64, vp, vp]
        L.wt_bitvector_rank.restype = ctypes.c_int
        L.wt_bitvector_select.argtypes = [vp, u64, u64, u32, vp, vp, vp, vp, u32, vp, vp, u64, vp, vp]
        L.wt_bitvector_select.restype = ctypes.c_int
        L.wt_alphabet.argtypes = [vp, u64, u32, vp, vp, ctypes.POINTER(u32), vp]
        L.wt_alphabet.restype = ctypes.c_int
        L.wt_train_select.argtypes = [vp, u32, ctypes.POINTER(TrainOptions), vp]
        L.wt_select_learned.argtypes = [vp, vp, vp, vp, u64, vp]
        L.wt_learned_info.argtypes = [vp, ctypes.POINTER(LearnedInfo)]
        fp = ctypes.POINTER(ctypes.c_float)
        L.wt_mlp_gradient.argtypes = [fp, fp, fp, u32, fp, fp]
        L.wt_batch_create.argtypes = [u32, ctypes.POINTER(vp), ctypes.POINTER(u64), ctypes.POINTER(u32), u32,
                                      ctypes.POINTER(BatchOptions), ctypes.POINTER(vp)]
        L.wt_batch_set_queries.argtypes = [vp, vp, vp, vp, vp, vp, u64]
        L.wt_batch_run.argtypes = [vp, vp]
        L.wt_batch_status_sync.argtypes = [vp, vp]
        L.wt_batch_tree.argtypes = [vp, u32, ctypes.POINTER(vp)]
        L.wt_batch_bytes.argtypes = [vp]
        L.wt_batch_bytes.restype = u64
        L.wt_batch_destroy.argtypes = [vp]
        L.wt_batch_destroy.restype = None
        L.wt_selftest_lookback_timeout.argtypes = [u32, vp]
        L.wt_selftest_lookback_timeout.restype = ctypes.c_int
        for f in ("wt_build", "wt_build_host", "wt_access", "wt_rank", "wt_select", "wt_query_mixed", "wt_query_host", "wt_status_sync",
                  "wt_info",
                  "wt_export", "wt_train_select", "wt_select_learned", "wt_learned_info", "wt_mlp_gradient",
                  "wt_batch_create", "wt_batch_set_queries", "wt_batch_run", "wt_batch_status_sync", "wt_batch_tree"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def status_str(s: int) -> str:
    return lib().wt_status_str(s).decode()


def _check(st: int, what: str):
    if st != WT_OK:
        raise WTError(st, what)


def _stream(stream=None) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _dptr(t, name):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _as_u64(t, name):
    import torch

    if t.dtype not in (torch.int64, getattr(torch, "uint64", torch.int64)):
        raise TypeError(f"{name} must be int64/uint64 (positions are 64-bit)")
    return _dptr(t, name)


def _as_u32(t, name):
    import torch

    if t.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)):
        raise TypeError(f"{name} must be int32/uint32")
    return _dptr(t, name)


class Tree:
    """Handle of a wavelet tree built on the GPU (wt_build)."""

    @classmethod
    def _view(cls, handle, n: int, sigma: int, symbol_bytes: int):
        t = cls.__new__(cls)
        t._h = handle
        t.n, t.sigma, t.symbol_bytes = n, sigma, symbol_bytes
        t._stream = None
        t.levels = t.info().levels
        return t

    def __init__(self, symbols, sigma: int, sample_k: int = 4096, stream=None, layout: int = 0,
                 allocator="torch"):
        import torch

        if symbols.dim() != 1:
            raise TypeError("symbols must be a 1-D tensor")
        w = symbols.element_size()
        if w not in (1, 2, 4) or symbols.dtype.is_floating_point:
            raise TypeError("symbols must be an integer tensor of 1, 2 or 4 bytes per element")
        self._keep = symbols.contiguous()
        self.n = symbols.numel()
        self.sigma = int(sigma)
        self.symbol_bytes = w
        self._stream = stream
        opt = Options(sample_k=sample_k, layout=layout)
        # tree memory from torch's caching allocator (default), a given
        # TorchAllocator / Allocator, or None for libwt's stream-ordered pool
        if isinstance(allocator, str) and allocator == "torch":
            allocator = torch_allocator()
        self._allocator = allocator
        if allocator is not None:
            st_ = allocator.struct if isinstance(allocator, TorchAllocator) else allocator
            opt.allocator = ctypes.pointer(st_)
        h = ctypes.c_void_p()
        ptr = self._keep.data_ptr() if self.n else None
        # a CPU tensor (pinned or pageable) goes through wt_build_host: chunked copy overlapping the histogram
        build_fn = lib().wt_build if symbols.is_cuda else lib().wt_build_host
        st = build_fn(ptr, self.n, self.sigma, w, ctypes.byref(opt), _stream(stream), ctypes.byref(h))
        self._keep = None  # the input is not retained after the call (it has synchronised once)
        _check(st, "wt_build")
        self._h = h
        self.levels = self.info().levels

    # ---- lifecycle ----
    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().wt_destroy(h)
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

    # ---- queries (outputs allocated with torch on the current device) ----
    def access(self, i, out=None, stream=None):
        import torch

        q = i.numel()
        if out is None:
            out = torch.empty(q, dtype=torch.int32, device=i.device)
        if q:
            _check(lib().wt_access(self._h, _as_u64(i, "i"), _dptr(out, "out"), q, _stream(stream)), "wt_access")
        return out

    def rank(self, c, i, out=None, stream=None):
        import torch

        q = i.numel()
        if c.numel() != q:
            raise ValueError("c and i must have the same length")
        if out is None:
            out = torch.empty(q, dtype=torch.int64, device=i.device)
        if q:
            _check(lib().wt_rank(self._h, _as_u32(c, "c"), _as_u64(i, "i"), _dptr(out, "out"), q, _stream(stream)),
                   "wt_rank")
        return out

    def select(self, c, j, out=None, stream=None):
        import torch

        q = j.numel()
        if c.numel() != q:
            raise ValueError("c and j must have the same length")
        if out is None:
            out = torch.empty(q, dtype=torch.int64, device=j.device)
        if q:
            _check(lib().wt_select(self._h, _as_u32(c, "c"), _as_u64(j, "j"), _dptr(out, "out"), q,
                                   _stream(stream)), "wt_select")
        return out

    def order(self, kind: int, arg, c=None, kinds=None, stream=None) -> "Order":
        """wt_order_queries: the batch (ORDER_ACCESS: arg = i; ORDER_RANK: c, i;
        ORDER_SELECT: c, j; ORDER_MIXED: kinds, c, arg) sorted by walk key into
        arrays the order owns, on `stream` (may differ from the build's, so the
        sort overlaps the level passes)."""
        return Order(self, kind, arg, c, kinds, stream)

    def walk(self, order: "Order", out=None, stream=None):
        """wt_walk_ordered: the order's answers, in the batch's original order."""
        import torch

        if out is None:
            out = torch.empty(order.q, dtype=torch.int32 if order.kind == ORDER_ACCESS else torch.int64,
                              device=order.device)
        if order.q:
            _check(lib().wt_walk_ordered(self._h, order._h, _dptr(out, "out"), _stream(stream)), "wt_walk_ordered")
        return out

    def query_mixed(self, kind, c, arg, out=None, stream=None):
        import torch

        q = arg.numel()
        if kind.numel() != q or c.numel() != q:
            raise ValueError("kind, c and arg must have the same length")
        if kind.dtype != torch.uint8:
            raise TypeError("kind must be uint8")
        if out is None:
            out = torch.empty(q, dtype=torch.int64, device=arg.device)
        if q:
            _check(lib().wt_query_mixed(self._h, _dptr(kind, "kind"), _as_u32(c, "c"), _as_u64(arg, "arg"),
                                        _dptr(out, "out"), q, _stream(stream)), "wt_query_mixed")
        return out

    def query_host(self, kind: int, arg, c=None, kinds=None, out=None, chunk: int = 0, stream=None):
        """wt_query_host: CPU tensors in (pinned or pageable), answers to the CPU
        tensor ``out`` (int32 for access, int64 otherwise).  Asynchronous: the
        answers are in ``out`` once ``stream`` has been synchronised."""
        import torch

        def host(t, name, dtypes):
            if not isinstance(t, torch.Tensor) or t.is_cuda:
                raise TypeError(f"{name} must be a CPU tensor")
            if t.dtype not in dtypes:
                raise TypeError(f"{name} has dtype {t.dtype}")
            if not t.is_contiguous():
                raise ValueError(f"{name} must be contiguous")
            return t.data_ptr()

        q = arg.numel()
        a = host(arg, "arg", (torch.int64, getattr(torch, "uint64", torch.int64)))
        cp = host(c, "c", (torch.int32, getattr(torch, "uint32", torch.int32))) if kind != 0 else None
        kp = host(kinds, "kinds", (torch.uint8,)) if kind == 3 else None
        for t, name in ((c, "c"), (kinds, "kinds")):
            if t is not None and t.numel() != q:
                raise ValueError(f"{name} and arg must have the same length")
        if out is None:
            out = torch.empty(q, dtype=torch.int32 if kind == 0 else torch.int64, pin_memory=True)
        if out.numel() != q:
            raise ValueError("out must have one entry per query")
        op = host(out, "out", (torch.int32,) if kind == 0 else (torch.int64,))
        if q:
            _check(lib().wt_query_host(self._h, kind, kp, cp, a, op, q, chunk, _stream(stream)), "wt_query_host")
        return out

    # ---- learned select ----
    def train_select(self, mode: int = LEARN_PLA, steps: int = 0, pairs: int = 0, lr: float = 0.0, stream=None):
        opt = TrainOptions(steps=steps, pairs=pairs, lr=lr)
        _check(lib().wt_train_select(self._h, mode, ctypes.byref(opt), _stream(stream)), "wt_train_select")

    def select_learned(self, c, j, out=None, stream=None):
        import torch

        q = j.numel()
        if c.numel() != q:
            raise ValueError("c and j must have the same length")
        if out is None:
            out = torch.empty(q, dtype=torch.int64, device=j.device)
        if q:
            _check(lib().wt_select_learned(self._h, _as_u32(c, "c"), _as_u64(j, "j"), _dptr(out, "out"), q,
                                           _stream(stream)), "wt_select_learned")
        return out

    def learned_info(self) -> LearnedInfo:
        inf = LearnedInfo()
        _check(lib().wt_learned_info(self._h, ctypes.byref(inf)), "wt_learned_info")
        return inf

    # ---- status / metadata ----
    def status_sync(self, stream=None) -> int:
        """Synchronise the stream; return and clear the sticky device status."""
        return lib().wt_status_sync(self._h, _stream(stream))

    def info(self) -> Info:
        inf = Info()
        _check(lib().wt_info(self._h, ctypes.byref(inf)), "wt_info")
        return inf

    def export(self, what: int, level: int = 0) -> np.ndarray:
        cnt = ctypes.c_uint64()
        _check(lib().wt_export(self._h, level, what, None, ctypes.byref(cnt)), "wt_export")
        dt = {EXPORT_L2: np.uint16, EXPORT_LENS: np.uint8, EXPORT_EPS0: np.uint32, EXPORT_EPS1: np.uint32,
              EXPORT_MLP: np.float32, EXPORT_RESID0: np.int32, EXPORT_RESID1: np.int32}.get(what, np.uint64)
        width = 4 if what == EXPORT_NODES else 1
        out = np.zeros(cnt.value * width, dt)
        if cnt.value:
            _check(lib().wt_export(self._h, level, what, out.ctypes.data, ctypes.byref(cnt)), "wt_export")
        return out.reshape(-1, 4) if what == EXPORT_NODES else out


def build(symbols, sigma: int, sample_k: int = 4096, stream=None, layout: int = LAYOUT_TREE,
          allocator="torch") -> Tree:
    """wt_build: construct the tree (or, with layout=LAYOUT_MATRIX, the wavelet
    matrix) of a 1-D CUDA tensor of symbols in [0, sigma); a CPU tensor goes
    through wt_build_host.  Device memory comes from torch's caching allocator
    unless ``allocator`` is None (libwt's pool) or another allocator."""
    return Tree(symbols, sigma, sample_k=sample_k, stream=stream, layout=layout, allocator=allocator)


class Batch:
    """Many independent trees built and queried by one CUDA graph launch (wt_batch_*).

    symbols: list of 1-D CUDA tensors (16-byte aligned, same element size); they
    must stay alive and unchanged in size while the batch exists."""

    def __init__(self, symbols, sigmas, sample_k: int = 4096, query_threads: int = 256, allocator=None,
                 lp_ctas_per_sm: int = 0):
        self._syms = list(symbols)
        nt = len(self._syms)
        w = self._syms[0].element_size()
        ptrs = (ctypes.c_void_p * nt)(*[t.data_ptr() if t.numel() else None for t in self._syms])
        ns = (ctypes.c_uint64 * nt)(*[t.numel() for t in self._syms])
        sg = (ctypes.c_uint32 * nt)(*[int(x) for x in sigmas])
        self.n = [t.numel() for t in self._syms]
        self.sigma = [int(x) for x in sigmas]
        self.symbol_bytes = w
        opt = BatchOptions(sample_k=sample_k, query_threads=query_threads, lp_ctas_per_sm=lp_ctas_per_sm)
        if isinstance(allocator, str) and allocator == "torch":
            allocator = torch_allocator()
        self._allocator = allocator
        if allocator is not None:
            opt.allocator = ctypes.pointer(allocator.struct if isinstance(allocator, TorchAllocator) else allocator)
        h = ctypes.c_void_p()
        _check(lib().wt_batch_create(nt, ptrs, ns, sg, w, ctypes.byref(opt), ctypes.byref(h)), "wt_batch_create")
        self._h = h
        self._q = None

    def set_queries(self, tree, kind, c, arg, out=None):
        import torch

        q = arg.numel()
        if out is None:
            out = torch.empty(q, dtype=torch.int64, device=arg.device)
        self._q = (tree, kind, c, arg, out)  # keep the buffers alive
        _check(lib().wt_batch_set_queries(self._h, _as_u32(tree, "tree"), _dptr(kind, "kind"), _as_u32(c, "c"),
                                          _as_u64(arg, "arg"), _dptr(out, "out"), q), "wt_batch_set_queries")
        return out

    def run(self, stream=None):
        _check(lib().wt_batch_run(self._h, _stream(stream)), "wt_batch_run")

    def status_sync(self, stream=None) -> int:
        return lib().wt_batch_status_sync(self._h, _stream(stream))

    def tree(self, i: int) -> "Tree":
        h = ctypes.c_void_p()
        _check(lib().wt_batch_tree(self._h, i, ctypes.byref(h)), "wt_batch_tree")
        return Tree._view(h, self.n[i], self.sigma[i], self.symbol_bytes)

    def nbytes(self) -> int:
        return int(lib().wt_batch_bytes(self._h))

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().wt_batch_destroy(h)
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


def alphabet(symbols, out=None, values: bool = True, stream=None):
    """wt_alphabet: (symbols mapped to [0, sigma) in the input's width, the
    distinct values in increasing order (uint32, or None), sigma)."""
    import torch

    w = {torch.uint8: 1, torch.int16: 2, torch.int32: 4}.get(symbols.dtype)
    if w is None:
        raise TypeError("symbols must be uint8, int16 or int32 (the bit patterns of u8/u16/u32 symbols)")
    n = symbols.numel()
    if out is None:
        out = torch.empty_like(symbols)
    vals = torch.empty(min(n, 1 << (8 * w)), dtype=torch.int32, device=symbols.device) if values and n else None
    sigma = ctypes.c_uint32(0)
    _check(lib().wt_alphabet(_dptr(symbols, "symbols") if n else None, n, w, _dptr(out, "out") if n else None,
                             vals.data_ptr() if vals is not None else None, ctypes.byref(sigma), _stream(stream)),
           "wt_alphabet")
    return out, (vals[: sigma.value] if vals is not None else None), sigma.value


class Bitvector:
    """A device bitvector (uint64 words, LSB-first) with its rank/select support,
    built by wt_bitvector_support_static; rank and select by wt_bitvector_rank /
    wt_bitvector_select.  The words are copied into an allocation padded to
    whole 512-bit blocks plus one."""

    def __init__(self, words, nbits: int, sample_k: int = 4096, stream=None):
        import torch

        if not isinstance(words, torch.Tensor) or not words.is_cuda or words.dtype != torch.int64:
            raise TypeError("words must be a CUDA int64 tensor")
        nw = (nbits + 63) // 64
        if words.numel() < nw:
            raise ValueError("words holds fewer than nbits bits")
        dev = words.device
        self.nbits, self.sample_k = nbits, sample_k
        self.words = torch.zeros((nbits // 512 + 1) * 8, dtype=torch.int64, device=dev)
        self.words[:nw] = words[:nw]
        if nbits % 64:
            self.words[nw - 1] &= (1 << (nbits % 64)) - 1
        self.l1 = torch.empty(nbits // 65536 + 1, dtype=torch.int64, device=dev)
        self.l2 = torch.empty(nbits // 512 + 1, dtype=torch.int16, device=dev)
        cap = nbits // sample_k + 2
        self.s0 = torch.empty(cap, dtype=torch.int64, device=dev)
        self.s1 = torch.empty(cap, dtype=torch.int64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self._ones = torch.zeros(1, dtype=torch.int64, device=dev)
        self._cap = cap
        self.support(stream)
        self.ones = int(self._ones.item())  # counted by the support kernel

    def support(self, stream=None):
        """wt_bitvector_support_static: (re)build the counters, samples and ones count."""
        _check(lib().wt_bitvector_support_static(self.words.data_ptr(), self.nbits, self.sample_k, self.l1.data_ptr(),
                                                 self.l2.data_ptr(), self.s0.data_ptr(), self.s1.data_ptr(),
                                                 self._cap, self.status.data_ptr(), self._ones.data_ptr(),
                                                 _stream(stream)),
               "wt_bitvector_support_static")

    def rank(self, i, out=None, stream=None):
        import torch

        q = i.numel()
        if out is None:
            out = torch.empty(q, dtype=torch.int64, device=i.device)
        _check(lib().wt_bitvector_rank(self.words.data_ptr(), self.nbits, self.l1.data_ptr(), self.l2.data_ptr(),
                                       _as_u64(i, "i"), _dptr(out, "out"), q, self.status.data_ptr(),
                                       _stream(stream)), "wt_bitvector_rank")
        return out

    def select(self, b: int, j, out=None, stream=None):
        import torch

        q = j.numel()
        if out is None:
            out = torch.empty(q, dtype=torch.int64, device=j.device)
        _check(lib().wt_bitvector_select(self.words.data_ptr(), self.nbits, self.ones, b, self.l1.data_ptr(),
                                         self.l2.data_ptr(), self.s0.data_ptr(), self.s1.data_ptr(), self.sample_k,
                                         _as_u64(j, "j"), _dptr(out, "out"), q, self.status.data_ptr(),
                                         _stream(stream)), "wt_bitvector_select")
        return out

    def status_sync(self) -> int:
        """Synchronise the device, return and clear the sticky status word."""
        import torch

        torch.cuda.synchronize()
        v = int(self.status.item())
        self.status.zero_()
        for code in (WT_EBOUNDS, WT_ETIMEOUT, WT_EQUERY):
            if v & (1 << code):
                return code
        return WT_OK


def mlp_gradient(params, u, t):
    """Loss and gradient of the learned-select MLP on the GPU (the training kernel's code)."""
    fp = ctypes.POINTER(ctypes.c_float)
    P = np.ascontiguousarray(params, np.float32)
    U = np.ascontiguousarray(u, np.float32)
    T = np.ascontiguousarray(t, np.float32)
    g = np.zeros(MLP_PARAMS, np.float32)
    loss = ctypes.c_float()
    _check(lib().wt_mlp_gradient(P.ctypes.data_as(fp), U.ctypes.data_as(fp), T.ctypes.data_as(fp), U.size,
                                 g.ctypes.data_as(fp), ctypes.byref(loss)), "wt_mlp_gradient")
    return g, float(loss.value)


# ---- launch accounting / kernel timing ----
def profile_enable(on: bool = True):
    lib().wt_profile_enable(1 if on else 0)


def profile_reset():
    lib().wt_profile_reset()


def profile_launches() -> int:
    return int(lib().wt_profile_launches())


def profile_report() -> dict:
    need = lib().wt_profile_report(None, 0)
    buf = ctypes.create_string_buffer(int(need) + 16)
    lib().wt_profile_report(buf, len(buf))
    return json.loads(buf.value.decode())
