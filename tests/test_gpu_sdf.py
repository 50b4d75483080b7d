"""GPU parity of the signed distance from clockwise line segments (Sec. 3.1,
mesh_segment_sdf_grid) with the oracle: bit-identical float32 values, on
every node of small grids and on sampled nodes of the 4096^2 grid."""
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


def _shapes():
    k = 720
    th = -2 * np.pi * np.arange(k) / k
    return {
        "star300": W.star_polygon(300, 0.4, 1.0, 5),
        "star500": W.star_polygon(500, 0.4, 1.0, 2),
        "L": np.array([[0, 0], [0, 2], [1, 2], [1, 1], [2, 1], [2, 0]], float) * 0.5 - 0.5,
        "square": np.array([[-0.5, -0.5], [-0.5, 0.5], [0.5, 0.5], [0.5, -0.5]]),
        "circle720": 0.8 * np.stack([np.cos(th), np.sin(th)], 1),
        "acute": np.array([[-1.0, -0.1], [-1.0, 0.1], [1.0, 0.0]]),
    }


@pytest.mark.parametrize("name", list(_shapes()))
def test_every_node_matches(name):
    import paper_2309_13824_gb300 as g

    v = _shapes()[name]
    n = 257
    got = g.segment_sdf_grid(v, n, BOX)
    X, Y = _nodes(n)
    want = oracle.segment_sdf(v, X.ravel(), Y.ravel()).reshape(n, n).astype(np.float32)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), np.count_nonzero(got != want)


def test_full_size_star_sampled():
    """The benchmark star's 4096^2 grid: 20,000 random nodes bit-identical,
    and the host-built grid of the workloads agrees wherever its sampled
    nearest-segment search found the closest segment."""
    import torch

    import paper_2309_13824_gb300 as g

    v = W.star_polygon(500, 0.4, 1.0, 2)
    n = 4096
    dev = torch.empty((n, n), dtype=torch.float32, device="cuda")
    g.segment_sdf_grid(v, n, BOX, out=dev)
    got = dev.cpu().numpy()
    rng = np.random.default_rng(3)
    i, j = rng.integers(0, n, 20000), rng.integers(0, n, 20000)
    x0, y0, x1, y1 = BOX
    px = x0 + i * ((x1 - x0) / (n - 1))
    py = y0 + j * ((y1 - y0) / (n - 1))
    want = oracle.segment_sdf(v, px, py).astype(np.float32)
    assert np.array_equal(got[j, i].view(np.uint32), want.view(np.uint32))
