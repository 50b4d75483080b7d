"""Pins of the FP64 reference of the learned model (oracle/mlp.py)."""
import numpy as np
import pytest

from oracle import mlp as M


def _batch(n=37, seed=0):
    rng = np.random.default_rng(seed)
    X = np.zeros((n, M.K_IN))
    X[:, : M.N_FEAT] = rng.standard_normal((n, M.N_FEAT))
    T = rng.standard_normal((n, M.N_OUT))
    return X, T


def test_gradients_match_finite_differences():
    X, T = _batch()
    P = M.Params.random(3)
    L, G = M.loss_and_grads(P, X, T, quantize=False)
    p0, g = P.flat(), G.flat()
    rng = np.random.default_rng(1)
    # every bias and a sample of the weights of each layer
    o1 = M.HID * M.K_IN
    o2 = o1 + M.HID + M.HID * M.HID
    o3 = o2 + M.HID + M.N_OUT * M.HID
    pick = np.concatenate([rng.choice(o1, 60, replace=False), np.arange(o1, o1 + M.HID),
                           rng.choice(np.arange(o1 + M.HID, o2), 60, replace=False), np.arange(o2, o2 + M.HID),
                           np.arange(o2 + M.HID, o3), np.arange(o3, M.N_PARAMS)])
    eps = 1e-6
    for k in pick:
        pp, pm = p0.copy(), p0.copy()
        pp[k] += eps
        pm[k] -= eps
        lp, _ = M.loss_and_grads(M.Params.from_flat(pp), X, T, quantize=False)
        lm, _ = M.loss_and_grads(M.Params.from_flat(pm), X, T, quantize=False)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])), (k, fd, g[k])


@pytest.mark.parametrize("quantize", [False, True])
def test_hand_computed_network(quantize):
    W1 = np.zeros((M.HID, M.K_IN))
    W1[0, 0] = 2.0
    W2 = np.zeros((M.HID, M.HID))
    W2[0, 0] = 3.0
    W3 = np.zeros((M.N_OUT, M.HID))
    W3[0, 0] = 0.5
    P = M.Params(W1, np.zeros(M.HID), W2, np.zeros(M.HID), W3, np.array([1.0, -1.0]))
    X = np.zeros((1, M.K_IN))
    X[0, 0] = 1.0
    Y, _ = M.forward(P, X, quantize)
    assert np.array_equal(Y, [[4.0, -1.0]])
    L, G = M.loss_and_grads(P, X, np.zeros((1, 2)), quantize)
    assert L == 8.5
    assert G.W3[0, 0] == 24.0 and G.W3[1, 0] == -6.0 and np.array_equal(G.b3, [4.0, -1.0])
    assert G.W2[0, 0] == 4.0 and G.b2[0] == 2.0 and np.count_nonzero(G.W2) == 1
    assert G.W1[0, 0] == 6.0 and G.b1[0] == 6.0 and np.count_nonzero(G.W1) == 1


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-8, -3.0 - 2**-7, 1e-3])
    r = M.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0  # tie to even
    assert r[2] == 1.0 + 2**-6  # above the tie
    assert r[3] == -3.0  # 2^-7 is half an ulp at 3: tie to even
    assert abs(r[4] - 1e-3) <= 2**-9 * 1e-3


def test_knn_against_kdtree():
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(4)
    p = rng.uniform(-1, 1, (300, 2))
    nb = M.knn(p)
    d, i = cKDTree(p).query(p, k=M.N_NEIGH + 1)
    assert np.array_equal(nb, i[:, 1:])


def test_knn_lattice_ties():
    # interior point of a square lattice: 4 neighbours at s, 4 at s sqrt 2,
    # 4 at 2s, then 4 of the 8 at s sqrt 5 (the smallest indices)
    s = 0.125
    g = np.array([(i * s, j * s) for j in range(9) for i in range(9)])
    c = 4 * 9 + 4
    nb = M.knn(g)[c]
    off = (g[nb] - g[c]) / s
    d2 = (off**2).sum(1)
    assert list(d2) == [1] * 4 + [2] * 4 + [4] * 4 + [5] * 4
    ring5 = [k for k in range(len(g)) if k != c and ((g[k] - g[c]) ** 2).sum() / s**2 == 5]
    assert sorted(nb[12:]) == sorted(ring5)[:4]
    assert list(nb[:4]) == sorted(nb[:4])  # equal distances: by index


def test_feature_invariances():
    import workloads as W

    rng = np.random.default_rng(6)
    # points on a dyadic grid, so translating and rotating are exact
    p = rng.integers(-512, 512, (200, 2)) / 1024.0
    p = np.unique(p, axis=0)
    h = np.full(len(p), 0.05)
    siz = W.constant_grid(0.05)
    bnd = np.zeros(len(p), bool)
    F = M.features(p, h, 0.05, siz, bnd, 0)
    Ft = M.features(p + np.array([0.25, -0.5]), h, 0.05, siz, bnd, 0)
    assert np.array_equal(F, Ft)
    Fr = M.features(np.stack([-p[:, 1], p[:, 0]], 1), h, 0.05, siz, bnd, 1)
    off, offr = F[:, :32].reshape(-1, 16, 2), Fr[:, :32].reshape(-1, 16, 2)
    d2 = (off**2).sum(-1)
    ok = np.all(np.diff(d2, axis=1) > 0, axis=1)  # no distance ties: same order after rotation
    assert ok.sum() > 100
    assert np.array_equal(offr[ok, :, 0], -off[ok, :, 1]) and np.array_equal(offr[ok, :, 1], off[ok, :, 0])
    assert np.all(Fr[:, 36] == 1) and np.all(F[:, 32] == 0) and np.all(F[:, 33:35] == 0)
    assert np.all(F[:, 37:] == 0)
    # the last move, relative to h
    Fm = M.features(p, h, 0.05, siz, bnd, 0, previous=p - np.array([0.0125, -0.025]))
    assert np.all(Fm[:, 37] == np.float32(0.25)) and np.all(Fm[:, 38] == np.float32(-0.5))


def test_sizing_gradient_of_a_linear_field():
    import workloads as W

    g = W.grid_from_fn(lambda x, y: 0.01 + 0.002 * x - 0.003 * y, 33)
    for x, y in [(0.1, 0.2), (-0.77, 0.5), (1.0, -1.05)]:
        gx, gy = M.sizing_gradient(g, x, y)
        assert abs(gx - 0.002) < 1e-7 and abs(gy + 0.003) < 1e-7
