"""GPU parity at the full sizes of the benchmark workloads, on sampled rows.

Each workload is built at its full size (N = 70,000 MNIST-shaped, 131,071
binary-tree diffusion, 1,000,000 single-cell-like, and the 64-embedding
batch), the context is set up as the benchmark sets it up (launch shapes
from the autotuner), and the gradient is compared with the FP64 oracle on
sampled rows: the oracle builds its own tree over all points, walks every
point for Z, and evaluates the sampled rows one by one.  Bars as in the
small-size tests: FP64 relative 1e-9, FP32-mixed relative L2 1e-3 (Z 1e-4)
and the per-row bar of bars.py.
The states are Y0 ~ N(0, 1e-4 I) (the protocol's start) and a synthetic
rim-heavy spread state; neither comes from the CUDA path.
"""
import numpy as np
import pytest

import oracle
from bars import FP32_ROW_TOL, FP32_TOL, FP64_TOL, rel, worst_row
from paper_2401_13708_gb300 import HyperbolicTSNE, inputs

pytestmark = pytest.mark.gpu

ROWS = 2000

_cache = {}


def workload(name):
    if name not in _cache:
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        w = inputs.make_workload(name, seed=0, device=dev)
        _cache[name] = (w, inputs.spread_embedding(w.labels, 0))
    return _cache[name]


def rows_for(n, seed=7):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(ROWS, n), replace=False))


def gpu_grad(precision, w, y, theta):
    with HyperbolicTSNE(precision=precision) as t:
        t.set_P(w.indptr, w.indices, w.values)
        t.set_Y(y)
        if theta > 0:
            t.autotune(theta, 2)
        return t.grad(theta, 1.0)


@pytest.mark.parametrize("name,theta,state", [
    ("mnist_like", 0.5, "y0"), ("mnist_like", 0.5, "spread"),
    ("binary_tree", 0.2, "spread"), ("binary_tree", 0.5, "spread"), ("binary_tree", 0.8, "spread"),
    ("single_cell", 0.5, "y0"), ("single_cell", 0.5, "spread"), ("single_cell", 0.8, "spread"),
])
def test_fullsize_fp32_sampled_rows(name, theta, state):
    w, spread = workload(name)
    y = w.y0 if state == "y0" else spread
    rows = rows_for(w.n)
    ref = oracle.bh_grad(y, w.indptr, w.indices, w.values, theta=theta, exag=1.0, rows=rows)
    g, Z = gpu_grad("fp32", w, y, theta)
    assert Z == pytest.approx(ref["Z"], rel=1e-4)
    assert rel(g[rows], ref["g"]) < FP32_TOL
    assert worst_row(g[rows], ref) < FP32_ROW_TOL


@pytest.mark.parametrize("name,theta", [("binary_tree", 0.2), ("binary_tree", 0.8), ("single_cell", 0.5)])
def test_fullsize_fp64_sampled_rows(name, theta):
    w, spread = workload(name)
    rows = rows_for(w.n, seed=11)
    ref = oracle.bh_grad(spread, w.indptr, w.indices, w.values, theta=theta, exag=1.0, rows=rows)
    g, Z = gpu_grad("fp64", w, spread, theta)
    assert Z == pytest.approx(ref["Z"], rel=1e-11)
    assert rel(g[rows], ref["g"]) < FP64_TOL


def test_fullsize_batched_segments():
    """All 64 embeddings in one context (FP32-mixed, autotuned shapes); four
    segments -- the smallest, the largest and two others -- against the oracle
    on the whole segment."""
    import torch
    w = inputs.make_batched(64, seed=0, device="cuda" if torch.cuda.is_available() else "cpu")
    off = w.extra["offsets"]
    sizes = np.diff(off)
    y = np.concatenate([inputs.spread_embedding(w.labels[off[s]:off[s + 1]], 100 + s)
                        for s in range(len(off) - 1)])
    with HyperbolicTSNE(precision="fp32") as t:
        t.set_P(w.indptr, w.indices, w.values)
        t.set_Y(y)
        t.set_segments(off)
        t.autotune(0.5, 2)
        g, _ = t.grad(0.5, 1.0)
        zs = t.segment_Z()
    pick = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 17, 42})
    for s in pick:
        a, b = int(off[s]), int(off[s + 1])
        e0, e1 = int(w.indptr[a]), int(w.indptr[b])
        ip = (w.indptr[a:b + 1] - e0).astype(np.int64)
        ix = (w.indices[e0:e1] - a).astype(np.int32)
        ref = oracle.bh_grad(y[a:b], ip, ix, w.values[e0:e1], theta=0.5, exag=1.0)
        assert zs[s] == pytest.approx(ref["Z"], rel=1e-4)
        assert rel(g[a:b], ref["g"]) < FP32_TOL
        assert worst_row(g[a:b], ref) < FP32_ROW_TOL
