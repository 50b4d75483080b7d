"""Independent exact brute-force Delaunay used to pin the oracle.

Pure Python with fractions.Fraction: no code shared with the oracle or the
CUDA path.  The symbolic perturbation is evaluated literally: the lifted
coordinate of point r is |p_r|^2 + delta^(id_r + 1) with a concrete tiny
delta, which reproduces the limit sign for the inputs used in the tests.
"""
from fractions import Fraction
from itertools import combinations

DELTA = Fraction(1, 2 ** 90)


def F(x):
    return Fraction(float(x))


def orient(a, b, c):
    return (F(b[0]) - F(a[0])) * (F(c[1]) - F(a[1])) - (F(b[1]) - F(a[1])) * (F(c[0]) - F(a[0]))


def det3(m):
    return (m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1])
            - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0])
            + m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]))


def det4_lifted(pts, ids=None):
    """det of rows [x, y, x^2 + y^2 (+ delta^(id+1)), 1]."""
    rows = []
    for k, p in enumerate(pts):
        x, y = F(p[0]), F(p[1])
        z = x * x + y * y
        if ids is not None:
            z += DELTA ** (ids[k] + 1)
        rows.append([x, y, z, Fraction(1)])
    # expand along last column
    total = Fraction(0)
    for r in range(4):
        minor = [[rows[i][j] for j in range(3)] for i in range(4) if i != r]
        total += (-1) ** (r + 3) * det3(minor)
    return total


def sign(x):
    return (x > 0) - (x < 0)


def incircle(a, b, c, d):
    return sign(det4_lifted([a, b, c, d]))


def incircle_sos(a, ia, b, ib, c, ic, d, idd):
    s = sign(det4_lifted([a, b, c, d]))
    if s:
        return s
    return sign(det4_lifted([a, b, c, d], [ia, ib, ic, idd]))


def delaunay(points):
    """All CCW triangles (i<j<k sorted to start at min id) whose perturbed
    circumcircle contains no other point."""
    n = len(points)
    out = []
    for i, j, k in combinations(range(n), 3):
        o = orient(points[i], points[j], points[k])
        if o == 0:
            continue
        a, b = (j, k) if o > 0 else (k, j)
        ok = True
        for l in range(n):
            if l in (i, j, k):
                continue
            # inside circle(i,a,b) (CCW) iff perturbed det4 > 0
            if incircle_sos(points[i], i, points[a], a, points[b], b, points[l], l) > 0:
                ok = False
                break
        if ok:
            out.append((i, a, b))
    return sorted(out)
