"""Training the learned displacement model on the method's own trajectories.

A mesh is stepped by the plain method; every `horizon` + 1 iterations the
features of all its points (including their last move) are recorded together
with the displacement the method then makes over the next `horizon`
iterations, divided by h_i (``Mesh.collect_pairs``, all on the device).  The model is fitted to these
pairs by the library's tensor-core forward/backward kernels and Adam
(``MLP.train``).  Applying it with ``Mesh.step_learned`` every `horizon`
iterations proposes that many iterations' worth of movement in one step; the
plain iterations that follow judge each proposal and undo the ones that lower
the mesh quality.
"""
from __future__ import annotations

from . import MLP, Mesh


def collect(sdf, sizing, xy, method=2, precision=0, horizon=10, max_snapshots=40, stream=None):
    """(X, T) device tensors of training pairs from one trajectory of the
    plain method started at xy, until it terminates or max_snapshots."""
    import torch

    m = Mesh(sdf, sizing, xy, method=method, precision=precision, stream=stream)
    n = len(xy)
    xs, ts = [], []
    for _ in range(max_snapshots):
        X = torch.empty((n, 48), dtype=torch.int16, device="cuda")
        T = torch.empty((n, 2), dtype=torch.float32, device="cuda")
        m.collect_pairs(horizon, X, T)
        xs.append(X)
        ts.append(T)
        if m.step(0)["terminated"]:
            break
    m.close()
    return torch.cat(xs), torch.cat(ts)


def train(trajectories, horizon=10, epochs=40, fine_epochs=10, batch=8192, lr=1e-3, seed=0, stream=None):
    """Collect pairs from each (sdf, sizing, xy, method, precision) and fit a
    fresh model; returns (model, last-epoch loss, number of pairs)."""
    import torch

    parts = [collect(s, z, p, method=mt, precision=pr, horizon=horizon, stream=stream)
             for s, z, p, mt, pr in trajectories]
    X = torch.cat([a for a, _ in parts])
    T = torch.cat([b for _, b in parts])
    del parts
    net = MLP(seed=seed, stream=stream)
    loss = net.train(X, T, epochs=epochs, batch=batch, lr=lr, seed=seed)
    if fine_epochs:
        loss = net.train(X, T, epochs=fine_epochs, batch=batch, lr=lr * 0.2, seed=seed + 1)
    return net, loss, X.shape[0]


def time_to_quality(sdf, sizing, xy, net=None, target=None, precision=0, n_iters=2000, stream=None, **policy):
    """Wall time (seconds, host clock around device-synchronised calls) and
    statistics of the hybrid method from xy until the minimum angle reaches
    `target` (or, without a target, until the method terminates); plain
    iterations, or learned proposals with ``Mesh.step_learned`` when a model
    is given."""
    import time

    import torch

    m = Mesh(sdf, sizing, xy, method=2, precision=precision, stream=stream)
    if target:
        m.set_quality_target(target)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = m.step(n_iters) if net is None else m.step_learned(net, n_iters, **policy)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    m.close()
    return dt, s


def bench_kernels(n=1 << 20, batch=1 << 17, seed=0):
    """One inference pass over n random feature rows and one training epoch
    in batches of `batch` (times the model's kernels on their own)."""
    import numpy as np
    import torch

    from . import bf16_bits

    rng = np.random.default_rng(seed)
    X = np.zeros((n, 48), np.float32)
    X[:, :39] = rng.standard_normal((n, 39)).astype(np.float32)
    Xd = torch.from_numpy(bf16_bits(X).view(np.int16)).cuda()
    Td = torch.from_numpy(rng.standard_normal((n, 2)).astype(np.float32)).cuda()
    net = MLP(seed=seed)
    Y = net.forward(Xd)
    loss = net.train(Xd, Td, epochs=1, batch=batch, lr=1e-3)
    torch.cuda.synchronize()
    return float(Y.abs().mean()), loss


if __name__ == "__main__":
    import sys

    if "--bench" in sys.argv:
        print("forward |Y| mean %.4f, epoch loss %.4f" % bench_kernels())
