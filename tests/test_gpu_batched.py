"""GPU parity of batched embeddings and of CUDA-graph replay.

Several independent embeddings share one context (hts_set_segments): each
segment must give what the same problem gives alone -- the oracle on that
segment's points and P block, and a single-embedding context -- with the bars
of the single-problem parity tests:
  * keys (low 58 bits) and the per-segment tree: bit-exact, midpoints 4 ulp;
  * HTS_FP64 gradient, Z, KL and steps: relative 1e-9 against the oracle;
  * HTS_FP32_MIXED gradient: relative L2 error <= 1e-3 against the oracle,
    and the per-row bar of bars.py.
Graph replay runs the same kernels with the same arguments, so positions
after graph-replayed steps equal the eagerly launched ones bit for bit.
"""
import numpy as np
import pytest

import oracle
from bars import FP32_ROW_TOL, FP32_TOL, FP64_TOL, rel, worst_row
from paper_2401_13708_gb300 import HtsError, HyperbolicTSNE, inputs

pytestmark = pytest.mark.gpu

SEG_MASK = np.uint64((1 << 58) - 1)


_cache = {}


def batch(name="spread"):
    """Five mixtures of 200..2500 points; `spread` places each one out in the disk."""
    if name in _cache:
        return _cache[name]
    w = inputs.make_batched(5, seed=3, n_lo=200, n_hi=2500, value_dtype=np.float64)
    off = w.extra["offsets"]
    if name == "spread":
        y = np.concatenate([inputs.spread_embedding(w.labels[off[s]:off[s + 1]], 10 + s, rho_hi=6.0 + s)
                            for s in range(len(off) - 1)])
    else:
        y = w.y0.copy()
    _cache[name] = (w, y)
    return w, y


def block(w, s):
    """CSR block of segment s, re-indexed from 0."""
    off = w.extra["offsets"]
    a, b = int(off[s]), int(off[s + 1])
    e0, e1 = int(w.indptr[a]), int(w.indptr[b])
    ip = (w.indptr[a:b + 1] - e0).astype(np.int64)
    ix = (w.indices[e0:e1] - a).astype(np.int32)
    return ip, ix, w.values[e0:e1]


def batched_ctx(precision, w, y, lr_scale=None, **kw):
    t = HyperbolicTSNE(precision=precision, **kw)
    t.set_P(w.indptr, w.indices, w.values)
    t.set_Y(y)
    t.set_segments(w.extra["offsets"], lr_scale)
    return t


def test_offsets_and_blocks_are_consistent():
    w, _ = batch()
    off = w.extra["offsets"]
    assert off[0] == 0 and off[-1] == w.n and np.all(np.diff(off) > 0)
    for s in range(len(off) - 1):
        ip, ix, v = block(w, s)
        assert ix.min() >= 0 and ix.max() < off[s + 1] - off[s]
        assert v.sum() == pytest.approx(1.0, rel=1e-12)


@pytest.mark.parametrize("name", ["spread", "init"])
def test_keys_per_segment_bit_exact(name):
    w, y = batch(name)
    off = w.extra["offsets"]
    with batched_ctx("fp64", w, y) as t:
        k, _ = t.get_keys()
    for s in range(len(off) - 1):
        ks = k[off[s]:off[s + 1]]
        assert np.all((ks >> np.uint64(58)) == s)
        ko, _ = oracle.keys(y[off[s]:off[s + 1]], 0)
        assert np.array_equal(ks & SEG_MASK, ko)


@pytest.mark.parametrize("rule", [0, 1])
def test_forest_is_the_per_segment_trees(rule):
    w, y = batch()
    off = w.extra["offsets"]
    with batched_ctx("fp32", w, y, split_rule=rule) as t:
        g = t.get_tree()
    pos = 0
    for s in range(len(off) - 1):
        o = oracle.tree_export(y[off[s]:off[s + 1]], rule, which=1)
        m = o["depth"].shape[0]
        sl = slice(pos, pos + m)
        for k in ("depth", "prefix", "count"):
            assert np.array_equal(g[k][sl], o[k]), (s, k)
        first = np.where(o["first"] >= 0, o["first"] + off[s], -1)
        assert np.array_equal(g["first"][sl], first)
        ulp = np.spacing(np.abs(o["ycell"]))
        assert np.all(np.abs(g["ycell"][sl] - o["ycell"]) <= 4 * ulp)
        fin = np.isfinite(o["rcell"])
        assert np.array_equal(fin, np.isfinite(g["rcell"][sl]))
        assert np.allclose(g["rcell"][sl][fin], o["rcell"][fin], rtol=1e-12, atol=0)
        pos += m
    assert pos == g["depth"].shape[0]


@pytest.mark.parametrize("theta", [0.0, 0.5, 0.8])
def test_gradient_fp64_per_segment(theta):
    w, y = batch()
    off = w.extra["offsets"]
    with batched_ctx("fp64", w, y) as t:
        g, _ = t.grad(theta, 12.0)
        zs = t.segment_Z()
    for s in range(len(off) - 1):
        ys = y[off[s]:off[s + 1]]
        ip, ix, v = block(w, s)
        if theta == 0.0:
            ref = oracle.exact_grad(ys, ip, ix, v, exag=12.0)
        else:
            ref = oracle.bh_grad(ys, ip, ix, v, theta=theta, exag=12.0)
        assert zs[s] == pytest.approx(ref["Z"], rel=1e-12)
        assert rel(g[off[s]:off[s + 1]], ref["g"]) < FP64_TOL


@pytest.mark.parametrize("name", ["spread", "init"])
@pytest.mark.parametrize("theta", [0.0, 0.5])
def test_gradient_fp32_per_segment(name, theta):
    w, y = batch(name)
    off = w.extra["offsets"]
    with batched_ctx("fp32", w, y) as t:
        g, _ = t.grad(theta, 1.0)
        zs = t.segment_Z()
    for s in range(len(off) - 1):
        ys = y[off[s]:off[s + 1]]
        ip, ix, v = block(w, s)
        if theta == 0.0:
            ref = oracle.exact_grad(ys, ip, ix, v, exag=1.0)
        else:
            ref = oracle.bh_grad(ys, ip, ix, v, theta=theta, exag=1.0)
        assert zs[s] == pytest.approx(ref["Z"], rel=1e-4)
        assert rel(g[off[s]:off[s + 1]], ref["g"]) < FP32_TOL
        assert worst_row(g[off[s]:off[s + 1]], ref) < FP32_ROW_TOL


def test_batched_equals_single_contexts_fp32():
    w, y = batch()
    off = w.extra["offsets"]
    with batched_ctx("fp32", w, y) as t:
        g, _ = t.grad(0.5, 1.0)
    for s in range(len(off) - 1):
        ip, ix, v = block(w, s)
        with HyperbolicTSNE(precision="fp32") as u:
            u.set_P(ip, ix, v)
            u.set_Y(y[off[s]:off[s + 1]])
            u.set_walk_split(0)
            gs, _ = u.grad(0.5, 1.0)
        assert rel(g[off[s]:off[s + 1]], gs) < 1e-5


def test_kl_per_segment():
    w, y = batch()
    off = w.extra["offsets"]
    for theta in (0.0, 0.5):
        with batched_ctx("fp64", w, y) as t:
            kls = t.kl_segments(theta)
            total = t.kl(theta)
        refs = []
        for s in range(len(off) - 1):
            ip, ix, v = block(w, s)
            refs.append(oracle.kl(y[off[s]:off[s + 1]], ip, ix, v, theta=theta))
        assert np.allclose(kls, refs, rtol=1e-10, atol=0)
        assert total == pytest.approx(sum(refs), rel=1e-10)


@pytest.mark.parametrize("theta", [0.0, 0.5])
def test_steps_fp64_per_segment_learning_rates(theta):
    """The paper's lr = n / 12000 per embedding: lr = 1 times lr_scale = n_s / 12000.

    Against the oracle over 2 steps: near the rim (the last segment reaches
    |y| ~ 0.9999) exaggerated steps amplify rounding ~1e3-fold per step, so after
    5 steps the GPU and the oracle differ by ~1e-9 even for the exact gradient.  Against a single-embedding context, which rounds alike, over
    5 steps.
    """
    w, y = batch()
    off = w.extra["offsets"]
    sizes = np.diff(off).astype(np.float64)
    for nst in (2, 5):
        with batched_ctx("fp64", w, y, lr_scale=sizes / 12000.0) as t:
            t.step(nst, theta, 12.0, 1.0, 0.5)
            yg = t.get_Y()
        for s in range(len(off) - 1):
            ip, ix, v = block(w, s)
            ys = y[off[s]:off[s + 1]]
            if nst == 2:
                yo, _, _ = oracle.step(ys, np.zeros_like(ys), ip, ix, v, nst, theta, 12.0, sizes[s] / 12000.0, 0.5)
                assert rel(yg[off[s]:off[s + 1]], yo) < FP64_TOL
            else:
                with HyperbolicTSNE(precision="fp64") as u:
                    u.set_P(ip, ix, v)
                    u.set_Y(ys)
                    u.set_walk_split(0)  # the batched walk is unsplit: same summation order
                    u.step(nst, theta, 12.0, sizes[s] / 12000.0, 0.5)
                    yu = u.get_Y()
                assert rel(yg[off[s]:off[s + 1]], yu) < FP64_TOL


def test_single_point_segments():
    """Segments of one point (empty P rows) get zero force and Z = 0."""
    w, y = batch()
    # move two points into segments of their own by cutting their P entries
    ip, ix, v = block(w, 0)
    ys0 = y[:int(w.extra["offsets"][1])]
    keep = np.ones(ys0.shape[0], bool)
    keep[:2] = False
    rows = np.repeat(np.arange(ys0.shape[0]), np.diff(ip))
    m = keep[rows] & keep[ix]
    ix2, v2, r2 = ix[m], v[m], rows[m]
    ip2 = np.zeros(ys0.shape[0] + 1, np.int64)
    np.add.at(ip2, r2 + 1, 1)
    ip2 = np.cumsum(ip2)
    with HyperbolicTSNE(precision="fp64") as t:
        t.set_P(ip2, ix2.astype(np.int32), v2)
        t.set_Y(ys0)
        t.set_segments([0, 1, 2, ys0.shape[0]])
        g, _ = t.grad(0.5, 1.0)
        zs = t.segment_Z()
    assert np.all(g[:2] == 0.0) and zs[0] == 0.0 and zs[1] == 0.0
    sub_ip = (ip2[2:] - ip2[2]).astype(np.int64)
    ref = oracle.bh_grad(ys0[2:], sub_ip, (ix2[ip2[2]:] - 2).astype(np.int32), v2[ip2[2]:], theta=0.5)
    assert rel(g[2:], ref["g"]) < FP64_TOL


def test_segment_errors_leave_one_segment():
    w, y = batch()
    off = w.extra["offsets"]
    with HyperbolicTSNE(precision="fp64") as t:
        t.set_P(w.indptr, w.indices, w.values)
        t.set_Y(y)
        g1, z1 = t.grad(0.5, 1.0)
        with pytest.raises(HtsError):  # P couples the first two segments
            t.set_segments([0, int(off[1]) // 2, w.n])
        with pytest.raises(HtsError):
            t.set_segments([0, 0, w.n])
        with pytest.raises(HtsError):
            t.set_segments([0, w.n - 1])
        with pytest.raises(HtsError):
            t.set_segments(np.linspace(0, w.n, 66).astype(np.int64))
        assert t.nseg == 1
        g2, z2 = t.grad(0.5, 1.0)
        assert np.array_equal(g1, g2) and z1 == z2
        t.set_segments(off)
        t.set_segments([0, w.n])  # back to one embedding
        g3, z3 = t.grad(0.5, 1.0)
        assert np.array_equal(g1, g3) and z1 == z3


@pytest.mark.parametrize("segmented", [False, True])
def test_graph_replay_is_bit_identical(segmented):
    w, y = batch()
    lr_scale = np.diff(w.extra["offsets"]).astype(np.float64) if segmented else None
    out = []
    for graphs in (False, True):
        with HyperbolicTSNE(precision="fp32") as t:
            t.set_P(w.indptr, w.indices, w.values)
            t.set_Y(y)
            if segmented:
                t.set_segments(w.extra["offsets"], lr_scale)
            t.set_graphs(graphs)
            lr = 1.0 / 12000.0 if segmented else w.n / 12000.0
            t.step(7, 0.5, 12.0, lr, 0.5)
            t.step(5, 0.5, 1.0, lr, 0.8)  # new arguments: a new capture
            t.step(3, 0.5, 1.0, lr, 0.8)  # the cached one
            out.append(t.get_Y())
    assert np.array_equal(out[0], out[1])


def test_graph_replay_multi_tile_sort():
    """A captured iteration whose key sort spans several one-sweep tiles (9000
    points: nine 1024-key tiles with look-back) replays bit-identically."""
    w = inputs.make_workload("gaussian_mixture", seed=6, n=9000)
    y = inputs.spread_embedding(w.labels, 6)
    out = []
    for graphs in (False, True):
        with HyperbolicTSNE(precision="fp32") as t:
            t.set_P(w.indptr, w.indices, w.values)
            t.set_Y(y)
            t.set_graphs(graphs)
            t.step(6, 0.5, 12.0, w.n / 12000.0, 0.5)
            out.append(t.get_Y())
    assert np.array_equal(out[0], out[1])


def test_cosne_term_per_segment():
    """With segments the CO-SNE term of each point uses its segment's size."""
    w, y = batch()
    off = w.extra["offsets"]
    rng = np.random.default_rng(5)
    xsq = rng.uniform(0.0, 4.0, size=w.n)
    l1, l2 = 0.7, 0.05
    with batched_ctx("fp64", w, y) as t:
        t.set_cosne(l1, l2, xsq)
        g, _ = t.grad(0.5, 1.0)
    for s in range(len(off) - 1):
        a, b = int(off[s]), int(off[s + 1])
        ip, ix, v = block(w, s)
        gk = oracle.bh_grad(y[a:b], ip, ix, v, theta=0.5, exag=1.0)["g"]
        ref = oracle.cosne_grad(y[a:b], xsq[a:b], l1, l2, gk)
        assert rel(g[a:b], ref) < FP64_TOL
