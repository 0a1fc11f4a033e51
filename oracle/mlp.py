"""FP64 reference of the learned-select network and predictors (test infrastructure only).

The network maps the within-segment fraction u of a rank to u + g(u), with
g(u) = b2 + sum_j w2[j] * relu(w1[j] * u + b1[j]), 32 hidden units, parameters
packed as {w1[32], b1[32], w2[32], b2}.  The loss is the mean squared error of
u + g(u) against the position fraction t.  Forward and backward passes are
written out by hand; the backward pass is pinned by central finite
differences in tests/test_oracle_pins.py.

The FP32 predictor (``predict_mlp_f32`` and its array form) repeats the
kernel's chain of correctly rounded operations; its fused multiply-add
(``fma_f32``) rounds once, and it is pinned by exact rational arithmetic, by
the FP64 forward pass within the FP32 error bound, and by hand-computed
values of a one-unit network (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import numpy as np

H = 32
NPARAM = 3 * H + 1


def unpack(P):
    P = np.asarray(P, np.float64)
    return P[:H], P[H:2 * H], P[2 * H:3 * H], P[3 * H]


def forward(P, u):
    w1, b1, w2, b2 = unpack(P)
    u = np.asarray(u, np.float64)
    a = np.outer(u, w1) + b1
    h = np.maximum(a, 0.0)
    return h @ w2 + b2, a, h


def loss_and_grad(P, u, t):
    """Mean squared error of u + g(u) against t, and its gradient (NPARAM values)."""
    u = np.asarray(u, np.float64)
    t = np.asarray(t, np.float64)
    w1, b1, w2, b2 = unpack(P)
    y, a, h = forward(P, u)
    r = u + y - t
    n = u.size
    loss = float(np.mean(r * r))
    e = 2.0 * r / n
    gw2 = h.T @ e
    gb2 = e.sum()
    de = np.outer(e, w2) * (a > 0)
    gw1 = (de * u[:, None]).sum(axis=0)
    gb1 = de.sum(axis=0)
    return loss, np.concatenate([gw1, gb1, gw2, [gb2]])


def finite_difference_grad(P, u, t, h=1e-6):
    P = np.asarray(P, np.float64).copy()
    g = np.zeros_like(P)
    for i in range(P.size):
        p0 = P[i]
        P[i] = p0 + h
        lp, _ = loss_and_grad(P, u, t)
        P[i] = p0 - h
        lm, _ = loss_and_grad(P, u, t)
        P[i] = p0
        g[i] = (lp - lm) / (2 * h)
    return g


def knots(samples, total, size, m, K):
    """Knots of segment m: (k0, x0), (k1, x1) from the select samples of one level and bit."""
    k0, x0 = m * K, int(samples[m])
    if (m + 1) * K <= total:
        return k0, (m + 1) * K, x0, int(samples[m + 1])
    return k0, total + 1, x0, int(size)


def predict_pla(kn, k):
    """Linear interpolation between the knots, in exact integer arithmetic."""
    k0, k1, x0, x1 = kn
    return x0 + ((k - k0) * (x1 - x0)) // (k1 - k0)


def fma_f32(a, b, c):
    """Fused multiply-add of float32 values rounded once to float32 (round to
    nearest, ties to even), as CUDA's __fmaf_rn computes it; elementwise.

    The product a*b of two float32 values is exact in float64 (at most 48
    significant bits).  The sum p + c is formed in float64 with round-to-odd:
    the round-to-nearest sum s and its exact error e (Knuth's TwoSum) give the
    exact value s + e; when e != 0 and s's last significand bit is even, s is
    replaced by its float64 neighbour towards e.  Rounding a round-to-odd value
    with at least two more significand bits (53 >= 24 + 2) to float32 equals
    rounding the exact value once (Boldo and Melquiond, "Emulation of FMA and
    correctly rounded sums: proved algorithms using rounding to odd", IEEE
    Trans. Computers 57(4), 2008).
    """
    a = np.asarray(a, np.float32).astype(np.float64)
    b = np.asarray(b, np.float32).astype(np.float64)
    c = np.asarray(c, np.float32).astype(np.float64)
    p = a * b
    s = p + c
    pv = s - c
    cv = s - pv
    e = (p - pv) + (c - cv)
    even = (s.view(np.int64) & 1) == 0
    fix = (e != 0) & even
    s_odd = np.where(fix, np.nextafter(s, np.where(e > 0, np.inf, -np.inf)), s)
    return s_odd.astype(np.float32)


def _mlp_h_f32(u, P):
    """u + g(u) in the kernel's FP32 operation order: a_j = fma(w1_j, u, b1_j),
    y = fma(w2_j, max(a_j, 0), y) for j = 0..31 starting at y = b2, then u + y."""
    P = np.asarray(P, np.float32)
    u = np.asarray(u, np.float32)
    y = np.full(u.shape, P[3 * H], np.float32)
    for j in range(H):
        a = fma_f32(P[j], u, P[H + j])
        y = fma_f32(P[2 * H + j], np.maximum(a, np.float32(0)), y)
    return (u + y).astype(np.float32)


def predict_mlp_f32(kn, k, P):
    """Position predicted by the network for rank k in segment kn, in the
    kernel's FP32 arithmetic: u = (k - k0) / (k1 - k0) rounded to float32,
    h = clamp(u + g(u), 0, 1), offset = trunc(float32(x1 - x0) * h), capped
    at x1 - x0."""
    k0, k1, x0, x1 = kn
    f = np.float32
    u = f(f(k - k0) / f(k1 - k0))
    hh = f(min(max(_mlp_h_f32(u, P)[()], f(0)), f(1)))
    span = x1 - x0
    off = int(f(f(span) * hh))
    return x0 + min(off, span)


def segment_knots_all(samples, total, size, K):
    """Knots (k0, k1, x0, x1) of every rank k = 1..total, as int64 arrays (as in ``knots``)."""
    k = np.arange(1, total + 1, dtype=np.int64)
    m = k // K
    samples = np.asarray(samples, np.int64)
    k0 = m * K
    x0 = samples[m]
    has_next = (m + 1) * K <= total
    k1 = np.where(has_next, (m + 1) * K, total + 1)
    x1 = np.where(has_next, samples[np.minimum(m + 1, samples.size - 1)], size)
    return k, m, k0, k1, x0, x1


def predict_pla_all(k, k0, k1, x0, x1):
    """``predict_pla`` for arrays of ranks."""
    return x0 + ((k - k0) * (x1 - x0)) // (k1 - k0)


def predict_mlp_f32_all(k, k0, k1, x0, x1, P):
    """``predict_mlp_f32`` for arrays of ranks (same rounding steps, elementwise)."""
    f = np.float32
    u = ((k - k0).astype(np.float32) / (k1 - k0).astype(np.float32)).astype(np.float32)
    hh = np.clip(_mlp_h_f32(u, P), f(0), f(1)).astype(np.float32)
    span = x1 - x0
    off = (span.astype(np.float32) * hh).astype(np.float32).astype(np.int64)
    return x0 + np.minimum(off, span)


# --------------------------------------------------------------------------
# piecewise-linear model with fitted knots (the learned select's first model)
#
# Anchor segment m of a level and bit value b covers the ranks k with
# floor(k / (A K)) = m (A = ANCHOR consecutive select samples per segment);
# its ends are the anchors (k0, x0) = (m A K, S_b[A m]) and (k1, x1) =
# ((m+1) A K, S_b[A (m+1)]), or (count_b + 1, size) for the last segment.
# Knot t (t = 0..4) sits at rank kappa_t = k0 + floor(t (k1 - k0) / 4)
# (kappa_4 = k1) and position x0 + floor(t (x1 - x0) / 4) + R_t, with the
# fitted residuals R_1..3 (bits, signed) and R_0 = R_4 = 0.  A rank k is
# predicted from the two knots around it, (ka, xa) and (kb, xb) with ka <= k
# < kb, as xa + floor((k - ka) (xb - xa) / (kb - ka)) in exact integers.
# Segments shorter than four ranks interpolate between the anchors alone.
# --------------------------------------------------------------------------

ANCHOR = 4
NKNOT = 3


def anchor_knots(samples, total, size, m, K, A=ANCHOR):
    """(k0, k1, x0, x1) of anchor segment m from the level's select samples."""
    KA = A * K
    k0, x0 = m * KA, int(samples[A * m])
    if (m + 1) * KA <= total:
        return k0, (m + 1) * KA, x0, int(samples[A * (m + 1)])
    return k0, total + 1, x0, int(size)


def spline_knots(kn, R):
    """Knot ranks kappa_0..4 and positions xi_0..4 of a segment with residuals R[0..2]."""
    k0, k1, x0, x1 = kn
    kap = [k0 + ((t * (k1 - k0)) >> 2) for t in range(4)] + [k1]
    xi = [x0] + [x0 + ((t * (x1 - x0)) >> 2) + int(R[t - 1]) for t in (1, 2, 3)] + [x1]
    return kap, xi


def interp(ka, kb, xa, xb, k):
    """xa + floor((k - ka) (xb - xa) / (kb - ka)), Python integers."""
    return xa + ((k - ka) * (xb - xa)) // (kb - ka)


def predict_spline(kn, R, k):
    """Prediction for rank k (knots must be non-decreasing)."""
    k0, k1, x0, x1 = kn
    if k1 - k0 < 4:
        return interp(k0, k1, x0, x1, k)
    kap, xi = spline_knots(kn, R)
    t = int(k >= kap[1]) + int(k >= kap[2]) + int(k >= kap[3])
    return interp(kap[t], kap[t + 1], xi[t], xi[t + 1], k)


def predict_spline_all(k, k0, k1, x0, x1, R):
    """predict_spline for arrays: k, k0, k1, x0, x1 int64 arrays, R (len, 3) int64."""
    k, k0, k1, x0, x1 = (np.asarray(a, np.int64) for a in (k, k0, k1, x0, x1))
    R = np.asarray(R, np.int64).reshape(-1, 3)
    span = k1 - k0
    kap = [k0 + ((t * span) >> 2) for t in range(4)] + [k1]
    xi = [x0] + [x0 + ((t * (x1 - x0)) >> 2) + R[:, t - 1] for t in (1, 2, 3)] + [x1]
    t = (k >= kap[1]).astype(np.int64) + (k >= kap[2]) + (k >= kap[3])
    short = span < 4
    t = np.where(short, 0, t)
    kap_a, xi_a = np.stack(kap), np.stack(xi)
    idx = np.arange(k.size)
    ka = np.where(short, k0, kap_a[t, idx])
    kb = np.where(short, k1, kap_a[t + 1, idx])
    xa = np.where(short, x0, xi_a[t, idx])
    xb = np.where(short, x1, xi_a[t + 1, idx])
    return xa + ((k - ka) * (xb - xa)) // np.maximum(kb - ka, 1)


def segment_anchor_all(samples, total, size, K, A=ANCHOR):
    """For every rank k = 1..total: k, its segment m and the segment's anchors."""
    k = np.arange(1, total + 1, dtype=np.int64)
    KA = A * K
    m = k // KA
    samples = np.asarray(samples, np.int64)
    k0 = m * KA
    x0 = samples[A * m]
    has_next = (m + 1) * KA <= total
    k1 = np.where(has_next, (m + 1) * KA, total + 1)
    x1 = np.where(has_next, samples[np.minimum(A * (m + 1), samples.size - 1)], size)
    return k, m, k0, k1, x0, x1


def fit_spline_lsq(kn, ks, pos):
    """Least-squares residuals R_1..3 (FP64) of one segment: minimise
    sum_k (base(k) + sum_t R_t phi_t(k) - pos(k))^2 over its ranks ks with
    positions pos, base the untrained model (the piecewise-linear curve through
    the knots with R = 0) and phi_t the hat function that is 1 at kappa_t and
    0 at the neighbouring knots (the normal equations, a 3x3 system)."""
    k0, k1, x0, x1 = kn
    ks = np.asarray(ks, np.float64)
    pos = np.asarray(pos, np.float64)
    if k1 - k0 < 4 or ks.size == 0:
        return np.zeros(3)
    kap, xi0 = spline_knots(kn, [0, 0, 0])
    kap = np.array(kap, np.float64)
    base = np.interp(ks, kap, np.array(xi0, np.float64))
    Phi = np.zeros((ks.size, 3))
    for t in (1, 2, 3):
        up = (ks >= kap[t - 1]) & (ks <= kap[t])
        dn = (ks > kap[t]) & (ks <= kap[t + 1])
        Phi[up, t - 1] = (ks[up] - kap[t - 1]) / (kap[t] - kap[t - 1])
        Phi[dn, t - 1] = (kap[t + 1] - ks[dn]) / (kap[t + 1] - kap[t])
    A = Phi.T @ Phi
    y = Phi.T @ (pos - base)
    if abs(np.linalg.det(A)) < 1e-12:
        return np.linalg.lstsq(A, y, rcond=None)[0]
    return np.linalg.solve(A, y)
