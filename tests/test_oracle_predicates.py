"""Pins for the oracle's exact predicates (orient2d, incircle, SoS).

Reference values come from exact rational arithmetic (fractions.Fraction) in
tests/bruteforce.py, not from the oracle.
"""
import numpy as np
import pytest

import bruteforce as bf


def _rand_pts(rng, k, scale=1.0):
    return [tuple(rng.uniform(-scale, scale, 2)) for _ in range(k)]


def test_incircle_convention(oracle_mod):
    # counter-clockwise unit triangle; centre of its circumcircle is inside
    a, b, c = (0.0, 0.0), (1.0, 0.0), (0.0, 1.0)
    assert oracle_mod.orient2d(a, b, c) == 1
    assert oracle_mod.incircle(a, b, c, (0.5, 0.5)) == 1
    assert oracle_mod.incircle(a, b, c, (2.0, 2.0)) == -1
    assert oracle_mod.incircle(a, b, c, (1.0, 1.0)) == 0  # cocircular
    assert bf.incircle(a, b, c, (0.5, 0.5)) == 1


def test_orient_random_and_near_degenerate(oracle_mod):
    rng = np.random.default_rng(11)
    for _ in range(300):
        a, b = _rand_pts(rng, 2)
        t = rng.uniform(-2, 2)
        # points on (or one ulp off) the line through a and b
        c = (a[0] + t * (b[0] - a[0]), a[1] + t * (b[1] - a[1]))
        c = (np.nextafter(c[0], rng.choice([-1, 1]) * np.inf) if rng.random() < 0.5 else c[0], c[1])
        assert oracle_mod.orient2d(a, b, c) == bf.sign(bf.orient(a, b, c))


def test_orient_wide_exponents(oracle_mod):
    rng = np.random.default_rng(12)
    for _ in range(100):
        pts = [(float(rng.uniform(-1, 1) * 10.0 ** rng.integers(-300, 5)),
                float(rng.uniform(-1, 1) * 10.0 ** rng.integers(-300, 5))) for _ in range(3)]
        assert oracle_mod.orient2d(*pts) == bf.sign(bf.orient(*pts))


def test_incircle_near_cocircular(oracle_mod):
    rng = np.random.default_rng(13)
    for _ in range(200):
        cx, cy, r = rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(0.1, 1)
        th = rng.uniform(0, 2 * np.pi, 4)
        pts = [(cx + r * np.cos(t), cy + r * np.sin(t)) for t in th]
        if rng.random() < 0.5:
            pts[3] = (np.nextafter(pts[3][0], np.inf), pts[3][1])
        assert oracle_mod.incircle(*pts) == bf.incircle(*pts)


def test_incircle_exact_lattice_and_tiny(oracle_mod):
    s = 0.0625
    sq = [(0.0, 0.0), (s, 0.0), (s, s), (0.0, s)]
    assert oracle_mod.incircle(*sq) == 0
    pts = [(1e-300, 0.0), (1.0, 1e-310), (0.5, 0.5 + 1e-17), (0.25, -1e-290)]
    assert oracle_mod.incircle(*pts) == bf.incircle(*pts)


def test_sos_matches_literal_perturbation(oracle_mod):
    rng = np.random.default_rng(14)
    s = 0.125
    base = [(i * s, j * s) for i in range(3) for j in range(3)]
    for _ in range(150):
        idx = rng.choice(len(base), 4, replace=False)
        ids = [int(x) for x in rng.permutation(40)[:4]]
        pts = [base[k] for k in idx]
        if bf.orient(pts[0], pts[1], pts[2]) == 0 and bf.orient(pts[0], pts[1], pts[3]) == 0:
            continue
        want = bf.incircle_sos(pts[0], ids[0], pts[1], ids[1], pts[2], ids[2], pts[3], ids[3])
        got = oracle_mod.incircle_sos(pts[0], ids[0], pts[1], ids[1], pts[2], ids[2], pts[3], ids[3])
        if want != 0:
            assert got == want


def test_sos_never_zero_on_cocircular(oracle_mod):
    s = 0.0625
    sq = [(0.0, 0.0), (s, 0.0), (s, s), (0.0, s)]
    for perm in [(0, 1, 2, 3), (3, 2, 1, 0), (1, 3, 0, 2)]:
        v = oracle_mod.incircle_sos(sq[0], perm[0], sq[1], perm[1], sq[2], perm[2], sq[3], perm[3])
        assert v in (-1, 1)
        # swapping two rows flips the perturbed determinant
        w = oracle_mod.incircle_sos(sq[1], perm[1], sq[0], perm[0], sq[2], perm[2], sq[3], perm[3])
        assert w == -v
