"""GPU parity of the Eq. 7 sizing field (mesh_sizing_field) with the oracle:
bit-identical float32 values at every node of small grids and at sampled
nodes of a large one."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

BOX = (-1.1, -1.1, 1.1, 1.1)


def _nodes(n, box=BOX):
    x0, y0, x1, y1 = box
    xs = x0 + np.arange(n) * ((x1 - x0) / (n - 1))
    ys = y0 + np.arange(n) * ((y1 - y0) / (n - 1))
    return np.meshgrid(xs, ys)


def _samples(k, seed):
    """Points along a star polygon's boundary with varied local feature sizes."""
    rng = np.random.default_rng(seed)
    v = W.star_polygon(200, 0.4, 1.0, seed)
    a, b = v, np.roll(v, -1, 0)
    t = rng.uniform(0, 1, k)
    seg = rng.integers(0, len(v), k)
    s = a[seg] + t[:, None] * (b[seg] - a[seg])
    return s, rng.uniform(2e-4, 0.05, k)


@pytest.mark.parametrize("K", [0.0, 0.05, 0.2])
def test_every_node_matches(K):
    import paper_2309_13824_gb300 as g

    s, lfs = _samples(3000, 4)
    n = 257
    got = g.sizing_field(s, lfs, K, n, BOX)
    X, Y = _nodes(n)
    want = oracle.sizing_field(s, lfs, K, X.ravel(), Y.ravel()).reshape(n, n).astype(np.float32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), np.count_nonzero(got != want)


def test_large_grid_sampled():
    import torch

    import paper_2309_13824_gb300 as g

    s, lfs = _samples(50000, 5)
    n = 1024
    dev = torch.empty((n, n), dtype=torch.float32, device="cuda")
    g.sizing_field(s, lfs, 0.1, n, BOX, out=dev)
    got = dev.cpu().numpy()
    rng = np.random.default_rng(6)
    i, j = rng.integers(0, n, 5000), rng.integers(0, n, 5000)
    x0, y0, x1, y1 = BOX
    px = x0 + i * ((x1 - x0) / (n - 1))
    py = y0 + j * ((y1 - y0) / (n - 1))
    want = oracle.sizing_field(s, lfs, 0.1, px, py).astype(np.float32)
    assert np.array_equal(got[j, i].view(np.uint32), want.view(np.uint32))
