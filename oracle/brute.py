"""Pure-Python brute force for tiny inputs (test infrastructure only).

These functions restate the definitions directly and build the tree the
textbook way (a pointer-based tree whose nodes are then concatenated level by
level, Section 5), so they pin the C oracle without sharing its method:
the C oracle derives each level from a counting sort by code prefix instead.
"""
from __future__ import annotations


def access(S, i):
    """Section 1: the value at position i."""
    return S[i]


def rank(S, c, i):
    """Section 1: occurrences of c in S[0, i)."""
    return sum(1 for j in range(i) if S[j] == c)


def select(S, c, j):
    """Section 1: position of the j-th (1-based) occurrence of c."""
    seen = 0
    for p, s in enumerate(S):
        if s == c:
            seen += 1
            if seen == j:
                return p
    raise ValueError("fewer than j occurrences")


def _prev_pow2(x):
    p = 1
    while p * 2 < x:
        p *= 2
    return p


def pointer_tree_levels(S, sigma):
    """Bit arrays per level of the reduced tree, built as a pointer-based tree.

    A node covers the symbol interval [a, b) and the subsequence of S with
    symbols in it; its bit for a symbol s is 1 iff s >= a + prevPow2(b - a);
    its children take the two subsequences.  Level d is the concatenation of
    the bit arrays of all depth-d nodes from left to right (the level-wise
    variant of Section 5).  Returns a list of lists of 0/1.
    """
    levels = []
    # visit level by level so each level is concatenated left to right
    frontier = [(list(S), 0, sigma)]
    d = 0
    while frontier:
        nxt = []
        for seq, a, b in frontier:
            if b - a < 2:
                continue
            mid = a + _prev_pow2(b - a)
            while len(levels) <= d:
                levels.append([])
            levels[d].extend(1 if s >= mid else 0 for s in seq)
            nxt.append(([s for s in seq if s < mid], a, mid))
            nxt.append(([s for s in seq if s >= mid], mid, b))
        frontier = nxt
        d += 1
    return levels


def counters(bits, K, l1=65536, l2=512):
    """L1, L2 counters and zero/one select samples of a bit list, by counting."""
    bits = [int(b) for b in bits]
    n = len(bits)
    prefix = [0] * (n + 1)
    for p, b in enumerate(bits):
        prefix[p + 1] = prefix[p] + b
    L1 = [prefix[k * l1] for k in range(n // l1 + 1)]
    L2 = [prefix[m * l2] - prefix[(m * l2 // l1) * l1] for m in range(n // l2 + 1)]
    s1, s0 = [0], [0]
    ones = zeros = 0
    for p, b in enumerate(bits):
        if b:
            ones += 1
            if ones % K == 0:
                s1.append(p)
        else:
            zeros += 1
            if zeros % K == 0:
                s0.append(p)
    return L1, L2, s0, s1


# --------------------------------------------------------------------------
# binary rank and select, one position at a time (Sections 4.1 and 4.2)
# --------------------------------------------------------------------------

def bv_rank(bits, i):
    """Section 4.1: the number of ones among the first i bits."""
    c = 0
    for k in range(i):
        c += 1 if bits[k] else 0
    return c


def bv_select(bits, b, j):
    """Section 4.2: the position of the j-th (1-based) bit equal to b."""
    seen = 0
    for k, x in enumerate(bits):
        if int(x) == b:
            seen += 1
            if seen == j:
                return k
    raise ValueError("fewer than j bits equal to b")


def matrix_levels(S, sigma):
    """Wavelet matrix levels by list manipulation: level l's bit of every
    symbol, then the symbols with bit 0 in order followed by those with bit 1."""
    L = (sigma - 1).bit_length() if sigma > 1 else 0
    seq = [int(x) for x in S]
    levels = []
    for l in range(L):
        sh = L - 1 - l
        levels.append([(x >> sh) & 1 for x in seq])
        seq = [x for x in seq if not (x >> sh) & 1] + [x for x in seq if (x >> sh) & 1]
    return levels
