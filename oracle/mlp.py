"""FP64 CPU reference of the learned displacement model (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs use this module.
The paper's method has no learned part; this is the plain definition the GPU
kernels are checked against:

* features of a point i (39 values, zero-padded to 48): the offsets of its 16
  nearest other points (by squared FP64 distance, ties by smaller index,
  nearest first) scaled by r_i = 1 / h_i (rounded once to FP64), h_i the
  geometry-cell size of its cell (Sec. 3.7);
  ln(h_i / h_avg); the gradient of the sizing field mu at p_i (derivative of
  the bilinear interpolant, Sec. 3.3 grid); 1 if the point is a boundary point;
  1 if the current move is CVD; its last move scaled by r_i (zero when not
  known).  Each feature is rounded to float32 and then to BF16 (round to
  nearest, ties to even);
* the network: Z1 = X W1^T + b1, H1 = relu(Z1), Z2 = H1 W2^T + b2,
  H2 = relu(Z2), Y = H2 W3^T + b3 (64 hidden units, 2 outputs: the proposed
  displacement divided by h_i);
* the loss: L = sum over samples and outputs of (Y - T)^2 / (2 B) for a batch
  of B samples, and its gradients by the chain rule.

With quantize=True every operand the tensor cores read is rounded to BF16
where the device rounds it (inputs, weights, H1, H2, dY, dZ2, dZ1); sums are
exact in FP64 here and FP32 on the device.  Pins (tests/test_oracle_mlp.py):
finite differences of the unquantized loss, a hand-computed tiny network, the
16-nearest-neighbour search against an independent sort, and invariances of
the features.
"""
from __future__ import annotations

import numpy as np

N_FEAT = 39
K_IN = 48
HID = 64
N_OUT = 2
N_NEIGH = 16


def bf16_round(x) -> np.ndarray:
    """Round to float32, then to the nearest BF16 (ties to even); returned as float64."""
    u = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32)).view(np.uint32)
    r = ((u >> 16) & 1) + 0x7FFF
    b = ((u.astype(np.uint64) + r) >> 16).astype(np.uint32) << 16
    return b.view(np.float32).astype(np.float64)


def knn(points: np.ndarray, k: int = N_NEIGH) -> np.ndarray:
    """Indices of the k nearest other points of every point, nearest first;
    ties (equal FP64 squared distances) broken by the smaller index.  Brute
    force, O(n^2): for the small inputs of the tests."""
    p = np.asarray(points, dtype=np.float64)
    n = len(p)
    out = np.full((n, k), -1, dtype=np.int64)
    idx = np.arange(n)
    for i in range(n):
        dx = p[:, 0] - p[i, 0]
        dy = p[:, 1] - p[i, 1]
        d2 = dx * dx + dy * dy
        order = np.lexsort((idx, d2))
        order = order[order != i][:k]
        out[i, : len(order)] = order
    return out


def sizing_gradient(grid, x: float, y: float):
    """Derivatives of the bilinear interpolant of a node grid at (x, y),
    with the cell clamped to the grid (same lookup as the value)."""
    nx, ny = grid.values.shape[1], grid.values.shape[0]
    dx = (grid.x1 - grid.x0) / (nx - 1)
    dy = (grid.y1 - grid.y0) / (ny - 1)
    tx = (x - grid.x0) / dx
    ty = (y - grid.y0) / dy
    fi, fj = np.floor(tx), np.floor(ty)
    i = 0 if not fi >= 0 else (nx - 2 if fi > nx - 2 else int(fi))
    j = 0 if not fj >= 0 else (ny - 2 if fj > ny - 2 else int(fj))
    fx = min(max(tx - i, 0.0), 1.0)
    fy = min(max(ty - j, 0.0), 1.0)
    v = grid.values
    v00, v10 = float(v[j, i]), float(v[j, i + 1])
    v01, v11 = float(v[j + 1, i]), float(v[j + 1, i + 1])
    gx = ((v10 - v00) + fy * ((v11 - v01) - (v10 - v00))) / dx
    gy = ((v01 - v00) + fx * ((v11 - v10) - (v01 - v00))) / dy
    return gx, gy


def features(points, h, havg, sizing, is_boundary, method_cvd: int, previous=None) -> np.ndarray:
    """(n, 48) features (unrounded FP64; the network reads bf16_round of them);
    `previous` are the positions before the last iteration (or None)."""
    p = np.asarray(points, dtype=np.float64)
    n = len(p)
    nb = knn(p)
    X = np.zeros((n, K_IN))
    for i in range(n):
        r = 1.0 / float(h[i])
        for k in range(N_NEIGH):
            j = nb[i, k]
            if j < 0:
                continue
            X[i, 2 * k] = np.float32((p[j, 0] - p[i, 0]) * r)
            X[i, 2 * k + 1] = np.float32((p[j, 1] - p[i, 1]) * r)
        X[i, 32] = np.float32(np.log(h[i] / havg))
        gx, gy = sizing_gradient(sizing, p[i, 0], p[i, 1])
        X[i, 33] = np.float32(gx)
        X[i, 34] = np.float32(gy)
        X[i, 35] = 1.0 if is_boundary[i] else 0.0
        X[i, 36] = float(method_cvd)
        if previous is not None:
            X[i, 37] = np.float32((p[i, 0] - previous[i, 0]) * r)
            X[i, 38] = np.float32((p[i, 1] - previous[i, 1]) * r)
    return X


class Params:
    """Network parameters in FP64 (weights as the device's FP32 masters)."""

    def __init__(self, W1, b1, W2, b2, W3, b3):
        self.W1 = np.asarray(W1, dtype=np.float64).reshape(HID, K_IN)
        self.b1 = np.asarray(b1, dtype=np.float64).reshape(HID)
        self.W2 = np.asarray(W2, dtype=np.float64).reshape(HID, HID)
        self.b2 = np.asarray(b2, dtype=np.float64).reshape(HID)
        self.W3 = np.asarray(W3, dtype=np.float64).reshape(N_OUT, HID)
        self.b3 = np.asarray(b3, dtype=np.float64).reshape(N_OUT)

    @staticmethod
    def random(seed: int, scale: float = 1.0) -> "Params":
        rng = np.random.default_rng(seed)
        return Params(rng.standard_normal((HID, K_IN)) * scale / np.sqrt(N_FEAT), rng.standard_normal(HID) * 0.1,
                      rng.standard_normal((HID, HID)) * scale / np.sqrt(HID), rng.standard_normal(HID) * 0.1,
                      rng.standard_normal((N_OUT, HID)) * scale / np.sqrt(HID), rng.standard_normal(N_OUT) * 0.1)

    def flat(self) -> np.ndarray:
        return np.concatenate([self.W1.ravel(), self.b1, self.W2.ravel(), self.b2, self.W3.ravel(), self.b3])

    @staticmethod
    def from_flat(v) -> "Params":
        v = np.asarray(v, dtype=np.float64)
        o = 0
        parts = []
        for shape in ((HID, K_IN), (HID,), (HID, HID), (HID,), (N_OUT, HID), (N_OUT,)):
            m = int(np.prod(shape))
            parts.append(v[o:o + m].reshape(shape))
            o += m
        return Params(*parts)


N_PARAMS = HID * K_IN + HID + HID * HID + HID + N_OUT * HID + N_OUT


def _q(x, quantize):
    return bf16_round(x) if quantize else np.asarray(x, dtype=np.float64)


def forward(P: Params, X, quantize: bool = True):
    """Outputs Y (n, 2) and the intermediate values of the pass."""
    X = _q(X, quantize)
    W1, W2, W3 = _q(P.W1, quantize), _q(P.W2, quantize), _q(P.W3, quantize)
    Z1 = X @ W1.T + P.b1
    H1 = _q(np.maximum(Z1, 0.0), quantize)
    Z2 = H1 @ W2.T + P.b2
    H2 = _q(np.maximum(Z2, 0.0), quantize)
    Y = H2 @ W3.T + P.b3
    return Y, (X, W1, W2, W3, Z1, H1, Z2, H2)


def loss_and_grads(P: Params, X, T, quantize: bool = True, scales: bool = False):
    """L = sum (Y - T)^2 / (2 B) and its gradients as a Params of the same
    shapes; with scales=True also a Params holding, for every gradient
    element, the sum of the absolute values of the products it adds up
    (the size its accumulation rounding is relative to)."""
    Y, (Xq, W1, W2, W3, Z1, H1, Z2, H2) = forward(P, X, quantize)
    B = len(Y)
    R = Y - np.asarray(T, dtype=np.float64)
    L = float((R * R).sum() / (2 * B))
    dY = _q(R / B, quantize)
    gW3 = dY.T @ H2
    gb3 = dY.sum(0)
    dZ2 = _q((dY @ W3) * (Z2 > 0), quantize)
    gW2 = dZ2.T @ H1
    gb2 = dZ2.sum(0)
    dZ1 = _q((dZ2 @ W2) * (Z1 > 0), quantize)
    gW1 = dZ1.T @ Xq
    gb1 = dZ1.sum(0)
    G = Params(gW1, gb1, gW2, gb2, gW3, gb3)
    if not scales:
        return L, G
    a = np.abs
    S = Params(a(dZ1).T @ a(Xq), a(dZ1).sum(0), a(dZ2).T @ a(H1), a(dZ2).sum(0), a(dY).T @ a(H2), a(dY).sum(0))
    return L, G, S


def adam_step(P: Params, G: Params, m, v, t: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step on the flat parameter vector; returns (P, m, v)."""
    p, g = P.flat(), G.flat()
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1**t)
    vh = v / (1 - b2**t)
    return Params.from_flat(p - lr * mh / (np.sqrt(vh) + eps)), m, v
