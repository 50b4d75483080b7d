"""The device's exact predicates (the decisions of the Voronoi clipping)
against the oracle's independent big-integer predicates, on generic,
near-degenerate and exactly degenerate inputs.  Calls the C ABI hook
mesh_exact_predicates."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _queries(seed=0):
    rng = np.random.default_rng(seed)
    Q, I = [], []
    # generic
    for _ in range(1500):
        Q.append(rng.uniform(-1, 1, (4, 2)))
    # near-cocircular: four points on a circle, some nudged by one ulp
    for _ in range(1500):
        c, r = rng.uniform(-1, 1, 2), rng.uniform(1e-3, 1)
        th = rng.uniform(0, 2 * np.pi, 4)
        p = c + r * np.stack([np.cos(th), np.sin(th)], 1)
        if rng.random() < 0.5:
            p[3, 0] = np.nextafter(p[3, 0], np.inf)
        Q.append(p)
    # near-collinear first three points
    for _ in range(1000):
        a, b = rng.uniform(-1, 1, (2, 2))
        t = rng.uniform(-2, 2)
        c = a + t * (b - a)
        c[1] = np.nextafter(c[1], rng.choice([-np.inf, np.inf])) if rng.random() < 0.5 else c[1]
        Q.append(np.stack([a, b, c, rng.uniform(-1, 1, 2)]))
    # exact lattice degeneracies (cocircular squares, collinear rows, duplicates)
    s = 2.0 ** -6
    base = np.array([(i * s, j * s) for i in range(4) for j in range(4)]) - 0.03
    for _ in range(2000):
        Q.append(base[rng.choice(len(base), 4, replace=rng.random() < 0.1)])
    for q in Q:
        I.append(rng.permutation(1000)[:4])
    return np.array(Q), np.array(I, dtype=np.int32)


def test_device_predicates_match_oracle():
    import oracle
    import paper_2309_13824_gb300 as g

    g.build()
    oracle.build()
    Q, I = _queries()
    o_dev, c_dev = g.mesh_exact_predicates(Q, I)
    o_ref = np.array([oracle.orient2d(q[0], q[1], q[2]) for q in Q])
    c_ref = np.array([oracle.incircle_sos(q[0], int(i[0]), q[1], int(i[1]), q[2], int(i[2]), q[3], int(i[3]))
                      for q, i in zip(Q, I)])
    assert np.array_equal(o_dev, o_ref), np.flatnonzero(o_dev != o_ref)[:10]
    # where the oracle reports 0 the four points are collinear (no SoS decision)
    m = c_ref != 0
    assert np.array_equal(c_dev[m], c_ref[m]), np.flatnonzero(c_dev[m] != c_ref[m])[:10]
    assert m.sum() > 0.9 * len(m)
