"""mesh_bucket_points_noalloc: the counting sort for callers that cannot
allocate device memory (their GPU memory belongs to another allocator, or
cudaMalloc's implicit synchronisation is not acceptable on their loop).  It
keeps its scratch in a fixed array inside the library; its results must equal
mesh_bucket_points (which takes a caller scratch buffer) call after call,
since the shared scratch keeps the previous call's contents."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BOX = (-1.1, -1.1, 1.1, 1.1)


def _run(g, torch, pts, nbx, nby, noalloc):
    n = len(pts)
    x = torch.tensor(pts[:, 0], device="cuda")
    y = torch.tensor(pts[:, 1], device="cuda")
    bs = torch.full((nbx * nby + 1,), -7, dtype=torch.int32, device="cuda")
    si = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    if noalloc:
        g.mesh_bucket_points_noalloc(x, y, n, BOX, nbx, nby, bs, si, st)
    else:
        scratch = torch.zeros(2 * n + nbx * nby + 1024, dtype=torch.int32, device="cuda")
        g.mesh_bucket_points(x, y, n, BOX, nbx, nby, bs, si, scratch, st)
    torch.cuda.synchronize()
    return bs.cpu().numpy(), si.cpu().numpy()[:n]


def _same(a, b):
    bs_a, si_a = a
    bs_b, si_b = b
    assert np.array_equal(bs_a, bs_b)
    # order inside a bucket is unspecified: compare each bucket's members
    for k in range(len(bs_a) - 1):
        lo, hi = bs_a[k], bs_a[k + 1]
        if hi > lo:
            assert np.array_equal(np.sort(si_a[lo:hi]), np.sort(si_b[lo:hi])), k


def test_noalloc_matches_allocating_entry_point_twice():
    torch = pytest.importorskip("torch")
    import paper_2309_13824_gb300 as g

    g.build()
    rng = np.random.default_rng(42)
    cases = [(rng.uniform(-1.1, 1.1, (200_003, 2)), 137, 91),
             (rng.uniform(-0.5, 0.9, (77_777, 2)), 40, 300)]
    for pts, nbx, nby in cases:  # two calls in a row through the shared scratch
        want = _run(g, torch, pts, nbx, nby, noalloc=False)
        got = _run(g, torch, pts, nbx, nby, noalloc=True)
        _same(got, want)
        assert np.array_equal(np.sort(got[1]), np.arange(len(pts)))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_2309_13824_gb300 as g

    g.build()
    L = g.lib()
    dummy = C.c_void_p(1)
    rc = L.mesh_bucket_points_noalloc(dummy, dummy, 3_000_000, *BOX, 100, 100, dummy, dummy, None)
    assert rc == g.TRIME_EINVAL
    assert "4194304" in g.mesh_last_error()


@pytest.mark.parametrize("n,nbx,nby", [
    # 2n + nb + nb/4096 + 1 == 4194304 exactly: key, rank, counts and the
    # tile sums fill the whole scratch
    (2_090_916, 1039, 12),
    # a bucket grid near its own cap (4096 x 1024) with few points: the tile
    # sums (1024 of them) sit at the end of the scratch
    (500, 2048, 2047),
    # no points: every bucket is empty
    (0, 7, 5),
])
def test_noalloc_edge_sizes(n, nbx, nby):
    torch = pytest.importorskip("torch")
    import paper_2309_13824_gb300 as g

    g.build()
    assert 2 * n + nbx * nby + nbx * nby // 4096 + 1 <= 4194304
    rng = np.random.default_rng(n + nbx)
    pts = rng.uniform(-1.1, 1.1, (n, 2))
    want = _run(g, torch, pts, nbx, nby, noalloc=False)
    for _ in range(2):  # twice in a row through the shared scratch
        got = _run(g, torch, pts, nbx, nby, noalloc=True)
        _same(got, want)
    assert np.array_equal(np.sort(got[1]), np.arange(n))
    if n == 0:
        assert not got[0].any()


def test_noalloc_rejects_one_past_the_limit():
    import paper_2309_13824_gb300 as g

    g.build()
    L = g.lib()
    dummy = C.c_void_p(1)
    # one point more than the case that fills the scratch exactly
    assert L.mesh_bucket_points_noalloc(dummy, dummy, 2_090_917, *BOX, 1039, 12, dummy, dummy, None) == g.TRIME_EINVAL
    # a bucket grid beyond 4096 x 1024
    assert L.mesh_bucket_points_noalloc(dummy, dummy, 1, *BOX, 4097, 1024, dummy, dummy, None) == g.TRIME_EINVAL
