"""CPU oracle for the level-wise wavelet tree (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it and
shares no code with it: the oracle is plain C (``wt_oracle.c``) plus the
pure-Python brute force in ``brute.py``.

``O1`` answers queries from their definitions (Section 1 of the paper);
``O2Tree`` is a naive level-wise tree with reduced codes that follows
Algorithms 3-8.  Both are pinned by ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wt_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_vp = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/liboracle.so`` with gcc."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_codes_split.argtypes = [ctypes.c_uint32, _u64p, _u8p, _u32p]
        L.orc_codes_alg3.argtypes = [ctypes.c_uint32, _u64p, _u8p, _u32p]
        L.orc_o1_build.argtypes = [_vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, _u64p, _u64p]
        L.orc_o1_access.argtypes = [_vp, ctypes.c_int, ctypes.c_uint64, _u64p, ctypes.c_uint64, _u32p]
        L.orc_o1_rank.argtypes = [_u64p, _u64p, ctypes.c_uint64, ctypes.c_uint32, _u32p, _u64p, ctypes.c_uint64, _u64p]
        L.orc_o1_select.argtypes = [_u64p, _u64p, ctypes.c_uint32, _u32p, _u64p, ctypes.c_uint64, _u64p]
        L.orc_o2_build.argtypes = [_vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
        L.orc_o2_build.restype = _vp
        L.orc_o2_build_mt.argtypes = [_vp, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int]
        L.orc_o2_build_mt.restype = _vp
        L.orc_o2_query_mt.argtypes = [_vp, ctypes.c_int, _u32p, _u64p, ctypes.c_uint64, _vp, ctypes.c_int]
        L.orc_o2_query_mt.restype = None
        L.orc_default_threads.argtypes = []
        L.orc_default_threads.restype = ctypes.c_int
        L.orc_o2_free.argtypes = [_vp]
        L.orc_o2_levels.argtypes = [_vp]
        L.orc_o2_levels.restype = ctypes.c_uint32
        for f in ("orc_o2_level_size", "orc_o2_level_ones"):
            getattr(L, f).argtypes = [_vp, ctypes.c_uint32]
            getattr(L, f).restype = ctypes.c_uint64
        L.orc_o2_rank_b.argtypes = [_vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64]
        L.orc_o2_rank_b.restype = ctypes.c_uint64
        L.orc_o2_select_b.argtypes = [_vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64]
        L.orc_o2_select_b.restype = ctypes.c_uint64
        L.orc_o2_node_start.argtypes = [_vp, ctypes.c_uint64, ctypes.c_uint32]
        L.orc_o2_node_start.restype = ctypes.c_uint64
        L.orc_o2_export.argtypes = [_vp, ctypes.c_uint32, ctypes.c_uint32, _vp]
        L.orc_o2_export.restype = ctypes.c_uint64
        L.orc_o2_access.argtypes = [_vp, _u64p, ctypes.c_uint64, _u32p]
        L.orc_o2_rank.argtypes = [_vp, _u32p, _u64p, ctypes.c_uint64, _u64p]
        L.orc_o2_select.argtypes = [_vp, _u32p, _u64p, ctypes.c_uint64, _u64p]
        _lib = L
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _sym(S: np.ndarray):
    S = np.ascontiguousarray(S)
    if S.dtype not in (np.uint8, np.uint16, np.uint32):
        raise TypeError("symbols must be uint8, uint16 or uint32")
    return S, S.dtype.itemsize


# --------------------------------------------------------------------------
# codes
# --------------------------------------------------------------------------

def codes_split(sigma: int):
    """Reduced codes by the recursive alphabet split (Section 5.1).

    Returns (code left-aligned in L bits, length, L)."""
    code = np.zeros(max(sigma, 1), np.uint64)
    ln = np.zeros(max(sigma, 1), np.uint8)
    L = ctypes.c_uint32()
    lib().orc_codes_split(sigma, _p(code, _u64p), _p(ln, _u8p), ctypes.byref(L))
    return code, ln, int(L.value)


def codes_alg3(sigma: int):
    """Algorithm 3 (createCodes) transcribed step by step."""
    code = np.zeros(max(sigma, 1), np.uint64)
    ln = np.zeros(max(sigma, 1), np.uint8)
    L = ctypes.c_uint32()
    lib().orc_codes_alg3(sigma, _p(code, _u64p), _p(ln, _u8p), ctypes.byref(L))
    return code, ln, int(L.value)


# --------------------------------------------------------------------------
# O1: definitional queries
# --------------------------------------------------------------------------

class O1:
    """Occurrence lists of S: access/rank/select straight from the definitions."""

    def __init__(self, S: np.ndarray, sigma: int):
        S, w = _sym(S)
        self.S, self.w, self.n, self.sigma = S, w, S.size, sigma
        self.C = np.zeros(sigma + 1, np.uint64)
        self.occ = np.zeros(max(S.size, 1), np.uint64)
        rc = lib().orc_o1_build(S.ctypes.data, w, S.size, sigma, _p(self.C, _u64p), _p(self.occ, _u64p))
        if rc != 0:
            raise ValueError("symbol >= sigma in input")

    def access(self, i):
        i = np.ascontiguousarray(i, np.uint64)
        out = np.empty(i.size, np.uint32)
        lib().orc_o1_access(self.S.ctypes.data, self.w, self.n, _p(i, _u64p), i.size, _p(out, _u32p))
        return out

    def rank(self, c, i):
        c = np.ascontiguousarray(c, np.uint32)
        i = np.ascontiguousarray(i, np.uint64)
        out = np.empty(i.size, np.uint64)
        lib().orc_o1_rank(_p(self.C, _u64p), _p(self.occ, _u64p), self.n, self.sigma, _p(c, _u32p), _p(i, _u64p), i.size, _p(out, _u64p))
        return out

    def select(self, c, j):
        c = np.ascontiguousarray(c, np.uint32)
        j = np.ascontiguousarray(j, np.uint64)
        out = np.empty(j.size, np.uint64)
        lib().orc_o1_select(_p(self.C, _u64p), _p(self.occ, _u64p), self.sigma, _p(c, _u32p), _p(j, _u64p), j.size, _p(out, _u64p))
        return out


# --------------------------------------------------------------------------
# O2: naive level-wise tree following Algorithms 3-8
# --------------------------------------------------------------------------

EXPORT_BITS, EXPORT_L1, EXPORT_L2, EXPORT_S0, EXPORT_S1, EXPORT_C, EXPORT_CODES, EXPORT_LENS, EXPORT_NODES = range(9)
_EXPORT_DTYPE = {0: np.uint64, 1: np.uint64, 2: np.uint16, 3: np.uint64, 4: np.uint64,
                 5: np.uint64, 6: np.uint64, 7: np.uint8, 8: np.uint64}


def default_threads() -> int:
    """Host threads the O2 build and the threaded query loops use by default
    (the online CPUs)."""
    return int(lib().orc_default_threads())


class O2Tree:
    """Naive level-wise wavelet tree (reduced codes, |L1| = 65536, |L2| = 512).

    ``threads``: host threads for the build's counting sorts (0: all online
    CPUs; inputs below 2^16 symbols use one).  The tree does not depend on it."""

    def __init__(self, S: np.ndarray, sigma: int, K: int = 4096, threads: int = 0):
        S, w = _sym(S)
        self._S = S
        self.n, self.sigma, self.K = S.size, sigma, K
        self._h = lib().orc_o2_build_mt(S.ctypes.data, w, S.size, sigma, K, threads)
        if not self._h:
            raise ValueError("symbol >= sigma in input (or sigma == 0)")
        self.L = int(lib().orc_o2_levels(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_o2_free(h)
            self._h = None

    def level_size(self, l):
        return int(lib().orc_o2_level_size(self._h, l))

    def level_ones(self, l):
        return int(lib().orc_o2_level_ones(self._h, l))

    def export(self, what: int, level: int = 0) -> np.ndarray:
        cnt = int(lib().orc_o2_export(self._h, level, what, None))
        dt = _EXPORT_DTYPE[what]
        width = 4 if what == EXPORT_NODES else 1
        out = np.zeros(cnt * width, dt)
        if cnt:
            lib().orc_o2_export(self._h, level, what, out.ctypes.data)
        return out.reshape(cnt, 4) if what == EXPORT_NODES else out

    def bits(self, level: int) -> np.ndarray:
        """Level bit array unpacked to one uint8 per bit (size_l entries)."""
        words = self.export(EXPORT_BITS, level)
        b = np.unpackbits(words.view(np.uint8), bitorder="little")
        return b[: self.level_size(level)]

    def rank_b(self, level, b, i):
        return int(lib().orc_o2_rank_b(self._h, level, b, i))

    def select_b(self, level, b, k):
        return int(lib().orc_o2_select_b(self._h, level, b, k))

    def node_start(self, c, level):
        return int(lib().orc_o2_node_start(self._h, c, level))

    def access(self, i):
        i = np.ascontiguousarray(i, np.uint64)
        out = np.empty(i.size, np.uint32)
        lib().orc_o2_access(self._h, _p(i, _u64p), i.size, _p(out, _u32p))
        return out

    def rank(self, c, i):
        c = np.ascontiguousarray(c, np.uint32)
        i = np.ascontiguousarray(i, np.uint64)
        out = np.empty(i.size, np.uint64)
        lib().orc_o2_rank(self._h, _p(c, _u32p), _p(i, _u64p), i.size, _p(out, _u64p))
        return out

    def select(self, c, j):
        c = np.ascontiguousarray(c, np.uint32)
        j = np.ascontiguousarray(j, np.uint64)
        out = np.empty(j.size, np.uint64)
        lib().orc_o2_select(self._h, _p(c, _u32p), _p(j, _u64p), j.size, _p(out, _u64p))
        return out

    def query_mt(self, kind: int, arg, c=None, threads: int = 0):
        """access (kind 0), rank (1) or select (2) over a batch split across
        host threads (0: all online CPUs); the same answers as the methods above."""
        arg = np.ascontiguousarray(arg, np.uint64)
        cc = np.ascontiguousarray(c if c is not None else np.zeros(arg.size), np.uint32)
        out = np.empty(arg.size, np.uint32 if kind == 0 else np.uint64)
        lib().orc_o2_query_mt(self._h, kind, _p(cc, _u32p), _p(arg, _u64p), arg.size, out.ctypes.data, threads)
        return out


# --------------------------------------------------------------------------
# standalone bitvectors: binary rank and select by definition
# --------------------------------------------------------------------------

def bv_rank(bits, i):
    """rank_1(B, i) (Section 4.1): ones in B[0, i), for each i in [0, len(B)].
    bits: 0/1 array.  Prefix sums of the bits, a library primitive."""
    pre = np.concatenate([[0], np.cumsum(np.asarray(bits, dtype=np.int64))])
    return pre[np.asarray(i, dtype=np.int64)].astype(np.uint64)


def bv_select(bits, b, j):
    """select_b(B, j) (Section 4.2): position of the j-th (1-based) bit equal to
    b, for each j in [1, count_b]."""
    pos = np.flatnonzero(np.asarray(bits) == b)
    return pos[np.asarray(j, dtype=np.int64) - 1].astype(np.uint64)


def bitvector_support(bits, K):
    """Rank counters and select samples of a bitvector by definition (Sections
    4.1 and 4.2), from its prefix sums (a library primitive): L1[k] = ones in
    B[0, 65536 k) for k <= n / 65536; L2[m] = ones in B[65536 floor(512 m /
    65536), 512 m) for m <= n / 512; S_b[0] = 0 and S_b[m] = position of the
    (m K)-th bit equal to b.  Returns (L1, L2, S0, S1) as uint64, uint16,
    uint64, uint64 arrays."""
    bits = np.asarray(bits).astype(np.uint8)
    n = bits.size
    pre = np.concatenate([[0], np.cumsum(bits, dtype=np.int64)])
    l1 = pre[np.arange(n // 65536 + 1) * 65536].astype(np.uint64)
    m = np.arange(n // 512 + 1) * 512
    l2 = (pre[m] - pre[(m // 65536) * 65536]).astype(np.uint16)
    out = [l1, l2]
    for b in (0, 1):
        pos = np.flatnonzero(bits == b)
        k = np.arange(1, pos.size // K + 1)
        out.append(np.concatenate([[0], pos[k * K - 1]]).astype(np.uint64))
    return tuple(out)


def alphabet_map(S):
    """Minimal alphabet (Section 6.2): the distinct values of S in increasing
    order and each symbol's rank among them (sorting, a library primitive)."""
    values, inv = np.unique(np.asarray(S), return_inverse=True)
    return inv.astype(np.int64), values


# --------------------------------------------------------------------------
# the wavelet matrix (the variant named as future work in Section 7)
# --------------------------------------------------------------------------

class OMatrix:
    """Wavelet matrix by definition: plain L-bit codes (L = ceil(lg sigma));
    level 0 holds S, B_l[i] = bit L-1-l of the level's i-th symbol, and level
    l+1 is level l stably partitioned by that bit, zeros first (a stable sort
    on one bit, a library primitive).  Rank counters and select samples follow
    Sections 4.1 and 4.2, computed from prefix sums."""

    def __init__(self, S: np.ndarray, sigma: int, K: int = 4096):
        self.L = int(sigma - 1).bit_length() if sigma > 1 else 0
        self.K = K
        seq = np.asarray(S).astype(np.int64)
        self.levels = []
        for l in range(self.L):
            bits = ((seq >> (self.L - 1 - l)) & 1).astype(np.uint8)
            self.levels.append(bits)
            seq = seq[np.argsort(bits, kind="stable")]

    def zeros(self, l):
        return int((self.levels[l] == 0).sum())

    def export(self, what: int, level: int = 0) -> np.ndarray:
        bits = self.levels[level]
        n = bits.size
        if what == 0:  # bits as LSB-first uint64 words
            pad = np.zeros((n + 63) // 64 * 64, np.uint8)
            pad[:n] = bits
            return np.packbits(pad, bitorder="little").view(np.uint64)
        if what in (1, 2, 3, 4):  # L1, L2, S0, S1
            return bitvector_support(bits, self.K)[what - 1]
        raise ValueError(what)
