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
