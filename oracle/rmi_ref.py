"""FP64 reference of the learned-index maths (two-stage recursive model index).

TEST INFRASTRUCTURE ONLY. The learned index is not part of the paper: it replaces the
search that assigns a flow record to a registered subnet (Sec. III.B.2.1, the step the
paper accelerates with its /24 hash table, Sec. IV.A.1) by a model that predicts the
position of the address among the sorted range starts, followed by an exact bounded
search (Kraska et al., "The Case for Learned Index Structures", SIGMOD 2018).

Model, as both the oracle and the library define it:
  xn   = float32(x) * 2^-32                               (x a uint32 address)
  root = linear:  float32(ra * xn + rb), one rounding per operation
         mlp:     sum_j w2_j * relu(w1_j * xn + b1_j) + b2  (1 -> H -> 1, FP32, j in order)
  leaf = clamp(floor(root), 0, L-1)
  d    = float32(int64(x) - int64(x0[leaf]))
  pred = float32(a[leaf] * d + b[leaf]),  pos = clamp(floor(pred), 0, n-1)
Training (mean squared error):
  root target  = true position * L / n;   leaf target = true position
  linear stage on standardised input z = (d - mu) / sigma:  yhat = w z + c
  gradients    dL/dw = 2/m sum (yhat - y) z,  dL/dc = 2/m sum (yhat - y)

Pins (tests/test_oracle_pins.py): the FP32 evaluation (xnorm, root_linear, root_mlp,
_clamp_floor, leaf_first_addresses, leaf_predict) and the endpoint error bound against
values worked out by hand in tests/golden/rmi_hand.json, including the FP32 rounding of x
and of d, keys that rounding sends to the next leaf, and the clamps at 0 and n-1; least
squares against numpy.polyfit; gradients against central finite differences.
"""
from __future__ import annotations

from typing import Dict, Tuple

import numpy as np

F32 = np.float32
TWO_M32 = F32(2.0 ** -32)


# ------------------------------------------------------------------ closed forms

def lstsq_line(x: np.ndarray, y: np.ndarray) -> Tuple[float, float]:
    """Least-squares line y ~ a x + b in FP64 by the normal equations (centred)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    if x.size == 0:
        return 0.0, 0.0
    mx, my = x.mean(), y.mean()
    sxx = np.sum((x - mx) ** 2)
    if sxx == 0.0:
        return 0.0, float(my)
    a = np.sum((x - mx) * (y - my)) / sxx
    return float(a), float(my - a * mx)


def linear_grad(w: float, c: float, z: np.ndarray, y: np.ndarray) -> Tuple[float, float, float]:
    """MSE loss and its gradient for yhat = w z + c, in FP64."""
    z = np.asarray(z, np.float64)
    y = np.asarray(y, np.float64)
    m = z.size
    r = w * z + c - y
    return float(np.mean(r * r)), float(2.0 / m * np.sum(r * z)), float(2.0 / m * np.sum(r))


def mlp_forward(p: Dict[str, np.ndarray], xn: np.ndarray) -> np.ndarray:
    h = np.maximum(np.outer(xn, p["w1"]) + p["b1"], 0.0)
    return h @ p["w2"] + p["b2"]


def mlp_loss_grad(p: Dict[str, np.ndarray], xn: np.ndarray, y: np.ndarray):
    """MSE loss of the 1 -> H -> 1 ReLU network and its gradient, FP64 backprop."""
    xn = np.asarray(xn, np.float64)
    y = np.asarray(y, np.float64)
    w1 = np.asarray(p["w1"], np.float64)
    b1 = np.asarray(p["b1"], np.float64)
    w2 = np.asarray(p["w2"], np.float64)
    b2 = float(p["b2"])
    m = xn.size
    pre = np.outer(xn, w1) + b1          # [m, H]
    h = np.maximum(pre, 0.0)
    out = h @ w2 + b2                    # [m]
    r = out - y
    loss = float(np.mean(r * r))
    g_out = 2.0 / m * r                  # dL/dout
    g_w2 = h.T @ g_out
    g_b2 = float(np.sum(g_out))
    g_h = np.outer(g_out, w2) * (pre > 0.0)
    g_w1 = g_h.T @ xn
    g_b1 = g_h.sum(axis=0)
    return loss, {"w1": g_w1, "b1": g_b1, "w2": g_w2, "b2": g_b2}


# ------------------------------------------------------- FP32 model evaluation

def xnorm(x: np.ndarray) -> np.ndarray:
    return (np.asarray(x, np.uint32).astype(F32) * TWO_M32).astype(F32)


def root_linear(ra: float, rb: float, x: np.ndarray, n_leaves: int) -> np.ndarray:
    xn = xnorm(x)
    r = (F32(ra) * xn).astype(F32)
    r = (r + F32(rb)).astype(F32)
    return _clamp_floor(r, n_leaves)


def root_mlp(p: Dict[str, np.ndarray], x: np.ndarray, n_leaves: int) -> np.ndarray:
    xn = xnorm(x)
    w1 = np.asarray(p["w1"], F32)
    b1 = np.asarray(p["b1"], F32)
    w2 = np.asarray(p["w2"], F32)
    acc = np.zeros(xn.shape, F32)
    for j in range(w1.size):
        pre = ((w1[j] * xn).astype(F32) + b1[j]).astype(F32)
        h = np.maximum(pre, F32(0.0))
        acc = (acc + (w2[j] * h).astype(F32)).astype(F32)
    acc = (acc + F32(p["b2"])).astype(F32)
    return _clamp_floor(acc, n_leaves)


def _clamp_floor(v: np.ndarray, n: int) -> np.ndarray:
    """floor(v) clamped to [0, n-1]; NaN and negatives give 0 (truncation is floor for
    v >= 0)."""
    out = np.zeros(v.shape, np.int64)
    ok = v >= 0
    out[ok] = np.minimum(v[ok], F32(n - 1)).astype(np.int64)
    return out


def leaf_predict(a: np.ndarray, b: np.ndarray, x0: np.ndarray, leaf: np.ndarray, x: np.ndarray,
                 n: int) -> np.ndarray:
    d = (np.asarray(x, np.int64) - np.asarray(x0, np.int64)[leaf]).astype(F32)
    p = (np.asarray(a, F32)[leaf] * d).astype(F32)
    p = (p + np.asarray(b, F32)[leaf]).astype(F32)
    return _clamp_floor(p, n)


# --------------------------------------------------------- error bound by endpoints

def leaf_first_addresses(ra: float, rb: float, n_leaves: int) -> np.ndarray:
    """first[l] = smallest address the monotone linear root sends to a leaf >= l
    (first[0] = 0, first[L] = 2^32), by bisection over [0, 2^32]."""
    targets = np.arange(n_leaves + 1)
    lo_b = np.zeros(n_leaves + 1, np.int64)
    hi_b = np.full(n_leaves + 1, 1 << 32, np.int64)
    for _ in range(34):
        mid = (lo_b + hi_b) // 2
        midc = np.minimum(mid, (1 << 32) - 1)
        r = root_linear(ra, rb, midc.astype(np.uint32), n_leaves)
        ge = (r >= targets) & (mid < (1 << 32))
        hi_b = np.where(ge, mid, hi_b)
        lo_b = np.where(ge, lo_b, mid + 1)
    first = hi_b
    first[0] = 0
    first[n_leaves] = 1 << 32
    return first


def eps_endpoints_linear(starts: np.ndarray, ra: float, rb: float, a, b, x0, n_leaves: int):
    """Per-leaf error bounds for a monotone model (ra >= 0 and every a >= 0).

    With a monotone root every leaf owns one interval of addresses; with a monotone leaf
    line the prediction is non-decreasing inside it, while the true position is constant
    on each range. So the largest under-prediction on a (range, leaf) piece is at the
    piece's first address and the largest over-prediction at its last one.
    Returns (eps_lo, eps_hi): pred - true <= eps_lo and true - pred <= eps_hi.
    """
    starts = np.asarray(starts, np.int64)
    n = starts.size
    assert ra >= 0 and np.all(np.asarray(a) >= 0)
    first = leaf_first_addresses(ra, rb, n_leaves)
    bounds = np.unique(np.concatenate([starts, first[1:n_leaves]]))
    bounds = bounds[bounds < (1 << 32)]
    seg_lo = bounds
    seg_hi = np.concatenate([bounds[1:], [1 << 32]]) - 1
    t = np.searchsorted(starts, seg_lo, side="right") - 1
    leaf = root_linear(ra, rb, seg_lo.astype(np.uint32), n_leaves)
    p_lo = leaf_predict(a, b, x0, leaf, seg_lo, n)
    p_hi = leaf_predict(a, b, x0, leaf, seg_hi, n)
    eps_lo = np.zeros(n_leaves, np.int64)
    eps_hi = np.zeros(n_leaves, np.int64)
    np.maximum.at(eps_lo, leaf, np.maximum(p_hi - t, 0))
    np.maximum.at(eps_hi, leaf, np.maximum(t - p_lo, 0))
    return eps_lo, eps_hi


# ------------------------------------------------- minimax leaves and split leaves
#
# A leaf's worst-case error over every address it owns is what the proven bound
# measures, so a leaf is fitted by minimising that error (a Chebyshev, or minimax, fit)
# rather than the mean squared error over sampled lookups. Inside a leaf the true
# position is a step function: constant t_k on each piece [dlo_k, dhi_k] of a range
# (offsets from the leaf's first address). For a line f(d) = a d + c with a >= 0, the
# largest under-prediction on a piece is at dlo_k and the largest over-prediction at
# dhi_k, so the fit minimises
#     E(a, c) = max( max_k (t_k - f(dlo_k)),  max_k (f(dhi_k) - t_k) ).
# For a fixed slope the best c centres the band: with G(a) = max_k (t_k - a dlo_k) and
# H(a) = min_k (t_k - a dhi_k), c = (G + H) / 2 and E = (G - H) / 2. G is convex and H
# concave in a, so E(a) is convex and a ternary search finds its minimum. Since
# E(a) >= a * w_max / 2 for the widest piece and E(0) = (t_max - t_min) / 2, the optimal
# slope lies in [0, (t_max - t_min) / w_max].
#
# A leaf whose fitted window (about 2E + 3 positions after rounding and the floor) exceeds
# a target is split into `count` equal sub-leaves of 2^shift addresses (the last one
# takes the remainder): the hybrid form of Kraska et al.'s index, which replaces a leaf
# whose error is too large, here with one more level of linear models. split[l] = ((count - 1) << 8) | shift
# for a split leaf, 0 otherwise; sub-leaves follow the L leaves in leaf order.

def minimax_line(dlo, dhi, t, iters: int = 200):
    """FP64 minimax line over pieces: returns (a, c, E) with a >= 0 minimising E."""
    dlo = np.asarray(dlo, np.float64)
    dhi = np.asarray(dhi, np.float64)
    t = np.asarray(t, np.float64)
    if t.size == 0:
        return 0.0, 0.0, 0.0

    def band(a):
        g = np.max(t - a * dlo)
        h = np.min(t - a * dhi)
        return g, h

    wmax = max(float(np.max(dhi - dlo)), 1.0)
    lo, hi = 0.0, float(t.max() - t.min()) / wmax
    for _ in range(iters):
        m1 = lo + (hi - lo) / 3.0
        m2 = hi - (hi - lo) / 3.0
        g1, h1 = band(m1)
        g2, h2 = band(m2)
        if g1 - h1 < g2 - h2:
            hi = m2
        else:
            lo = m1
    a = (lo + hi) / 2.0
    g, h = band(a)
    return a, (g + h) / 2.0, (g - h) / 2.0


def interval_pieces(starts: np.ndarray, F: int, G: int):
    """Pieces of the ranges inside addresses [F, G): offsets from F and positions."""
    starts = np.asarray(starts, np.int64)
    n = starts.size
    if F >= G:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0, np.int64)
    i0 = int(np.searchsorted(starts, F, side="right") - 1)
    i1 = int(np.searchsorted(starts, G - 1, side="right") - 1)
    idx = np.arange(i0, i1 + 1)
    s = starts[idx]
    e = np.where(idx + 1 < n, starts[np.minimum(idx + 1, n - 1)], 1 << 32)
    return np.maximum(s, F) - F, np.minimum(e, G) - 1 - F, idx


def fit_interval_minimax(starts: np.ndarray, F: int, G: int):
    """Minimax leaf line for addresses [F, G) in the library's convention: x0 = F,
    pos = floor(a d + b) with b = c + 0.5 (the floor then rounds to the nearest position).
    Returns (a, b, E)."""
    dlo, dhi, t = interval_pieces(starts, F, G)
    if t.size == 0:
        return 0.0, 0.0, 0.0
    a, c, E = minimax_line(dlo, dhi, t)
    return a, c + 0.5, E


def split_tables(ra: float, rb: float, n_leaves: int, split: np.ndarray):
    """Leaf first addresses and, per model (L leaves then the sub-leaves in leaf order),
    its first address and the address one past its last; split leaves own no interval
    themselves (lo = hi)."""
    split = np.asarray(split, np.int64)
    first = leaf_first_addresses(ra, rb, n_leaves)
    count = np.where(split != 0, (split >> 8) + 1, 0)
    M = n_leaves + int(count.sum())
    lo = np.zeros(M, np.int64)
    hi = np.zeros(M, np.int64)
    lo[:n_leaves] = first[:n_leaves]
    hi[:n_leaves] = first[1:]
    nxt = n_leaves
    for l in np.nonzero(split)[0]:
        sh = int(split[l] & 0xFF)
        c = int(count[l])
        F, G = int(first[l]), int(first[l + 1])
        j = np.arange(c)
        lo[nxt:nxt + c] = F + (j << sh)
        hi[nxt:nxt + c] = np.minimum(F + ((j + 1) << sh), G)
        hi[nxt + c - 1] = G
        hi[l] = lo[l]
        nxt += c
    return first, lo, hi


def route_models(ra: float, rb: float, n_leaves: int, split: np.ndarray, first: np.ndarray,
                 x: np.ndarray) -> np.ndarray:
    """Model of each address: the root's leaf, or for a split leaf its sub-leaf
    j = min(((x - x0) mod 2^32) >> shift, count - 1) with x0 the leaf's first address."""
    split = np.asarray(split, np.int64)
    x = np.asarray(x, np.int64)
    leaf = root_linear(ra, rb, x.astype(np.uint32), n_leaves)
    model = leaf.copy()
    count = np.where(split != 0, (split >> 8) + 1, 0)
    base = n_leaves + np.concatenate([[0], np.cumsum(count)[:-1]])
    sp = split[leaf] != 0
    if np.any(sp):
        l = leaf[sp]
        x0 = np.minimum(first[l], (1 << 32) - 1)
        j = ((x[sp] - x0) & 0xFFFFFFFF) >> (split[l] & 0xFF)
        model[sp] = base[l] + np.minimum(j, count[l] - 1)
    return model


def eps_endpoints_models(starts: np.ndarray, ra: float, rb: float, n_leaves: int, split: np.ndarray,
                         a, b, x0):
    """eps_endpoints_linear for a model with split leaves: every model (leaf or sub-leaf)
    owns one interval of addresses under the monotone linear root, so the same endpoint
    argument gives each model's bounds. Returns (eps_lo, eps_hi) over all models (0 for
    split leaves)."""
    starts = np.asarray(starts, np.int64)
    n = starts.size
    assert ra >= 0 and np.all(np.asarray(a) >= 0)
    first, mlo, _ = split_tables(ra, rb, n_leaves, split)
    M = mlo.size
    bounds = np.unique(np.concatenate([starts, mlo, first[1:n_leaves]]))
    bounds = bounds[bounds < (1 << 32)]
    seg_lo = bounds
    seg_hi = np.concatenate([bounds[1:], [1 << 32]]) - 1
    t = np.searchsorted(starts, seg_lo, side="right") - 1
    model = route_models(ra, rb, n_leaves, split, first, seg_lo)
    p_lo = leaf_predict(a, b, x0, model, seg_lo, n)
    p_hi = leaf_predict(a, b, x0, model, seg_hi, n)
    eps_lo = np.zeros(M, np.int64)
    eps_hi = np.zeros(M, np.int64)
    np.maximum.at(eps_lo, model, np.maximum(p_hi - t, 0))
    np.maximum.at(eps_hi, model, np.maximum(t - p_lo, 0))
    return eps_lo, eps_hi
