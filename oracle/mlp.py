"""FP64 reference of the learned-select network and predictors (test infrastructure only).

The network maps the within-segment fraction u of a rank to u + g(u), with
g(u) = b2 + sum_j w2[j] * relu(w1[j] * u + b1[j]), 32 hidden units, parameters
packed as {w1[32], b1[32], w2[32], b2}.  The loss is the mean squared error of
u + g(u) against the position fraction t.  Forward and backward passes are
written out by hand; the backward pass is pinned by central finite
differences in tests/test_oracle_pins.py.
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


def predict_mlp_f32(kn, k, P):
    """The same prediction in emulated FP32 (products and sums rounded to float32 at each step)."""
    k0, k1, x0, x1 = kn
    f = np.float32
    P = np.asarray(P, np.float32)
    u = f(f(k - k0) / f(k1 - k0))
    y = P[3 * H]
    for j in range(H):
        a = f(np.float64(P[j]) * np.float64(u) + np.float64(P[H + j]))
        y = f(np.float64(P[2 * H + j]) * np.float64(max(a, f(0))) + np.float64(y))
    hh = f(min(max(f(u + y), f(0)), f(1)))
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
    P = np.asarray(P, np.float32)
    u = (f(1) * (k - k0).astype(np.float32)) / (k1 - k0).astype(np.float32)
    u = u.astype(np.float32)
    u64 = u.astype(np.float64)
    y = np.full(u.shape, P[3 * H], np.float32)
    for j in range(H):
        a = (np.float64(P[j]) * u64 + np.float64(P[H + j])).astype(np.float32)
        y = (np.float64(P[2 * H + j]) * np.maximum(a, f(0)).astype(np.float64) + y.astype(np.float64)).astype(np.float32)
    hh = np.clip((u + y).astype(np.float32), f(0), f(1)).astype(np.float32)
    span = x1 - x0
    off = (span.astype(np.float32) * hh).astype(np.float32).astype(np.int64)
    return x0 + np.minimum(off, span)
