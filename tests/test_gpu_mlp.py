"""Learned displacement model on the tensor cores vs the FP64 CPU oracle.

The tensor-core tile (tcgen05 MMAs on BF16 operands, FP32 accumulation in
tensor memory) must equal the exact product of the same BF16 values up to
FP32 accumulation rounding.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import paper_2309_13824_gb300 as g

    g.build()


@pytest.mark.parametrize("M,N,K", [(128, 16, 16), (256, 64, 48), (128, 256, 256), (384, 48, 64), (128, 80, 32)])
def test_tensor_core_tile(M, N, K):
    import paper_2309_13824_gb300 as g

    rng = np.random.default_rng(M + N + K)
    A = g.bf16_bits(rng.standard_normal((M, K)))
    B = g.bf16_bits(rng.standard_normal((N, K)))
    D = g.mesh_tc_gemm_bf16(A, B)
    a = g.bf16_to_float(A).astype(np.float64)
    b = g.bf16_to_float(B).astype(np.float64)
    exact = a @ b.T
    scale = np.abs(a) @ np.abs(b).T
    assert np.all(np.abs(D - exact) <= 2e-6 * scale + 1e-30), np.max(np.abs(D - exact) / scale)


def _features_like(n, seed):
    """Random inputs shaped like the features (39 used columns, zero padding)."""
    rng = np.random.default_rng(seed)
    X = np.zeros((n, 48))
    X[:, :32] = rng.standard_normal((n, 32)) * 1.5
    X[:, 32] = rng.uniform(-2, 2, n)
    X[:, 33:35] = rng.standard_normal((n, 2)) * 0.05
    X[:, 35] = rng.integers(0, 2, n)
    X[:, 36] = rng.integers(0, 2, n)
    X[:, 37:39] = rng.standard_normal((n, 2)) * 0.2
    return X


def _device_params(seed):
    from oracle import mlp as M

    P = M.Params.random(seed)
    p32 = P.flat().astype(np.float32)
    return M.Params.from_flat(p32.astype(np.float64)), p32


def test_forward_matches_oracle():
    import paper_2309_13824_gb300 as g
    from oracle import mlp as M

    P, p32 = _device_params(5)
    net = g.MLP(p32)
    assert np.array_equal(net.params(), p32)
    X = _features_like(1000, 1)
    Y = net.forward(g.bf16_bits(X)).astype(np.float64)
    Yo, (_, _, _, W3, _, _, _, H2) = M.forward(P, X, quantize=True)
    # scale of each output: the magnitudes its last sum is made of
    scale = np.abs(H2) @ np.abs(W3).T + np.abs(P.b3)
    err = np.abs(Y - Yo) / scale
    # FP32 sums vs exact ones, and rare one-ulp BF16 rounding flips of a hidden unit
    assert np.quantile(err, 0.99) < 1e-5, np.quantile(err, 0.99)
    assert err.max() < 2e-2, err.max()


def test_gradients_match_oracle():
    import paper_2309_13824_gb300 as g
    from oracle import mlp as M

    P, p32 = _device_params(7)
    net = g.MLP(p32)
    X = _features_like(700, 2)
    T = np.random.default_rng(3).standard_normal((700, 2)) * 0.5
    loss, grad = net.loss_grad(g.bf16_bits(X), T.astype(np.float32))
    Lo, Go = M.loss_and_grads(P, X, T.astype(np.float32).astype(np.float64), quantize=True)
    assert loss == pytest.approx(Lo, rel=1e-4)
    go = Go.flat()
    for name, a, b in (("W1", 0, 3072), ("b1", 3072, 3136), ("W2", 3136, 7232), ("b2", 7232, 7296),
                       ("W3", 7296, 7424), ("b3", 7424, 7426)):
        d = np.linalg.norm(grad[a:b] - go[a:b]) / np.linalg.norm(go[a:b])
        assert d < 1e-2, (name, d)


def test_training_reduces_loss():
    import torch

    import paper_2309_13824_gb300 as g

    # a smooth target of the inputs: the network must fit it on the device
    X = _features_like(20000, 4)
    T = np.stack([np.tanh(X[:, 0] - 0.5 * X[:, 3]), 0.3 * X[:, 1] * X[:, 2]], 1) * 0.5
    Xd = torch.from_numpy(g.bf16_bits(X).view(np.int16)).cuda()
    Td = torch.from_numpy(T.astype(np.float32)).cuda()
    net = g.MLP(seed=1)
    l0, _ = net.loss_grad(g.bf16_bits(X), T.astype(np.float32))
    l1 = net.train(Xd, Td, epochs=30, batch=1024, lr=2e-3)
    l2, _ = net.loss_grad(g.bf16_bits(X), T.astype(np.float32))
    assert l2 < 0.1 * l0, (l0, l1, l2)


@pytest.mark.parametrize("which", ["disk", "annulus"])
def test_features_match_oracle(which):
    import oracle
    import paper_2309_13824_gb300 as g
    from gpu_helpers import annulus_small, disk_small, h_of_points
    from oracle import mlp as M

    oracle.build()
    sdf, siz, pts = disk_small(n=3001, seed=3) if which == "disk" else annulus_small(n=2500, seed=5)
    method = 0 if which == "disk" else 1
    gm = g.Mesh(sdf, siz, pts, method=method)
    Xg, hg = gm.features()
    om = oracle.OracleMesh(sdf, siz, pts, method=method)
    h = h_of_points(om, pts)
    _, _, _, havg = om.geometry()
    Xo = g.bf16_bits(M.features(pts, h, havg, siz, om.classes() == 1, method))
    assert np.allclose(hg, h, rtol=1e-7)
    same = Xg == Xo
    assert same[:, :32].mean() > 0.9999 and same[:, 33:].all(), (same[:, :32].mean(), same[:, 33:].mean())
    assert same[:, 32].mean() > 0.999
    # any difference is one BF16 ulp (a division or logarithm rounded differently)
    d = np.abs(Xg.astype(np.int32) - Xo.astype(np.int32))
    assert d.max() <= 1


def test_learned_proposals_reach_the_target():
    # trained on the method's own trajectories (a disk with DistMesh, an
    # annulus with the hybrid), applied to annuli drawn with other seeds: the
    # iterations to the plain method's converged minimum angle minus 1 degree.
    # The gain of one training varies (the trajectories the pairs come from
    # are not bit-reproducible): totals of 130, 162 and 220 against the plain
    # 161 were seen with the same code.  The test asserts what every training
    # must do -- reach the target on every seed, keep some proposals, never be
    # far slower -- and the benchmark measures the gain over seeds.
    import workloads as W
    from paper_2309_13824_gb300 import learn

    disk = W.disk_workload(n=10000)
    ann = W.annulus_workload(n=200000, seed=11)
    net, loss, npairs = learn.train([(disk.sdf, disk.sizing, disk.points, 0, 0),
                                     (ann.sdf, ann.sizing, ann.points, 2, 0)], epochs=30, fine_epochs=5)
    assert npairs > 10**6 and loss < 0.01
    its_plain = its_learned = 0
    for seed in (21, 22, 23):
        wl = W.annulus_workload(n=200000, seed=seed)
        _, conv = learn.time_to_quality(wl.sdf, wl.sizing, wl.points)
        q = conv["min_angle_deg"] - 1.0
        _, sp = learn.time_to_quality(wl.sdf, wl.sizing, wl.points, target=q)
        _, sl = learn.time_to_quality(wl.sdf, wl.sizing, wl.points, net=net, target=q)
        assert sp["target_reached"] and sl["target_reached"], (seed, sp, sl)
        assert sl["accepted"] > 0
        its_plain += sp["iterations"]
        its_learned += sl["iterations"]
        print(f"seed {seed}: plain {sp['iterations']} iterations, learned {sl['iterations']} "
              f"({sl['accepted']} proposals kept, {sl['rejected']} undone)")
    assert its_learned < 1.5 * its_plain, (its_learned, its_plain)
