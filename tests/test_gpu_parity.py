"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars (from the arithmetic each path uses):
  * keys, tree structure (depth, key prefix, N_cell, leaf points): bit-exact;
  * cell midpoints: within 4 ulp (both sides round the same correctly rounded
    sums through the same float64 formula);
  * HTS_FP64 gradient, Z, KL and 10 steps of positions: relative 1e-9;
  * HTS_FP32_MIXED gradient: relative L2 error <= 1e-3 against the oracle at
    the same theta (the paper's own BH-vs-exact error is 1e-3 .. 2.7e-3), and
    every row within 1e-3 of the size of its two force terms (bars.py).
Sizes span several 32-point warps, 256-thread blocks and 4096-key sort
tiles, with ragged tails.
"""
import math

import numpy as np
import pytest

import oracle
from bars import FP32_ROW_TOL, FP32_TOL, FP64_TOL, maxrel, rel, worst_row
from paper_2401_13708_gb300 import HyperbolicTSNE, inputs

pytestmark = pytest.mark.gpu


def make(precision, w, y, **kw):
    t = HyperbolicTSNE(precision=precision, **kw)
    t.set_P(w.indptr, w.indices, w.values)
    t.set_Y(y)
    return t


_cache = {}


def workload(name):
    if name in _cache:
        return _cache[name]
    if name == "mixture":
        w = inputs.make_workload("gaussian_mixture", seed=0)
        y = inputs.spread_embedding(w.labels, 0, rho_hi=8.0)
    elif name == "mixture_init":
        w = inputs.make_workload("gaussian_mixture", seed=0)
        y = w.y0
    elif name == "ragged":
        w = inputs.make_workload("gaussian_mixture", seed=4, n=4097)
        y = inputs.spread_embedding(w.labels, 4)
    elif name == "tree_small":
        w = inputs.make_workload("binary_tree", seed=0, n=8191)
        y = inputs.spread_embedding(w.labels, 1, rho_hi=10.0)
    elif name == "mnist_small":
        w = inputs.make_workload("mnist_like", seed=0, n=12000)
        y = inputs.spread_embedding(w.labels, 2, rho_hi=12.0)
    else:
        raise KeyError(name)
    _cache[name] = (w, y)
    return w, y


@pytest.mark.parametrize("name", ["mixture", "mixture_init", "ragged"])
@pytest.mark.parametrize("rule", [0, 1])
def test_keys_bit_exact(name, rule):
    w, y = workload(name)
    with make("fp64", w, y, split_rule=rule) as t:
        k, b = t.get_keys()
    ko, bo = oracle.keys(y, rule)
    assert np.array_equal(b, bo)
    assert np.array_equal(k, ko)


@pytest.mark.parametrize("name", ["mixture", "mixture_init", "ragged", "tree_small"])
@pytest.mark.parametrize("rule", [0, 1])
def test_tree_matches_oracle(name, rule):
    w, y = workload(name)
    with make("fp32", w, y, split_rule=rule) as t:
        g = t.get_tree()
    o = oracle.tree_export(y, rule, which=1)
    for k in ("depth", "prefix", "count", "first"):
        assert np.array_equal(g[k], o[k]), k
    ulp = np.spacing(np.abs(o["ycell"]))
    assert np.all(np.abs(g["ycell"] - o["ycell"]) <= 4 * ulp)
    fin = np.isfinite(o["rcell"])
    assert np.array_equal(fin, np.isfinite(g["rcell"]))
    assert np.allclose(g["rcell"][fin], o["rcell"][fin], rtol=1e-12, atol=0)


@pytest.mark.parametrize("n", [4096, 4097, 196608, 196609, 524288, 524289])
def test_tree_across_sort_paths(n):
    """The key sort runs in one block up to 4096 keys and as one-sweep passes
    with decoupled look-back above, in tiles of 1024 keys up to 196,608 keys,
    2048 up to 524,288 and 8192 (512 threads) beyond; both sides of every
    boundary build the oracle's tree.  (P plays no part in the tree: it is
    empty here.)"""
    labels = (np.arange(n) * 7919) % 37
    y = inputs.spread_embedding(labels, n % 5, rho_hi=10.0)
    with HyperbolicTSNE(precision="fp32") as t:
        t.set_P(np.zeros(n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
        t.set_Y(y)
        g = t.get_tree()
    o = oracle.tree_export(y, 0, which=1)
    for k in ("depth", "prefix", "count", "first"):
        assert np.array_equal(g[k], o[k]), k


@pytest.mark.parametrize("name", ["mixture", "mixture_init", "ragged"])
def test_exact_fp64(name):
    w, y = workload(name)
    ref = oracle.exact_grad(y, w.indptr, w.indices, w.values, exag=12.0)
    with make("fp64", w, y) as t:
        g, Z = t.grad(0.0, 12.0)
    assert Z == pytest.approx(ref["Z"], rel=1e-12)
    assert rel(g, ref["g"]) < FP64_TOL
    assert maxrel(g, ref["g"]) < FP64_TOL


@pytest.mark.parametrize("name", ["mixture", "mixture_init", "ragged", "tree_small"])
@pytest.mark.parametrize("theta", [0.2, 0.5, 0.8])
def test_bh_fp64(name, theta):
    w, y = workload(name)
    ref = oracle.bh_grad(y, w.indptr, w.indices, w.values, theta=theta, exag=1.0)
    with make("fp64", w, y) as t:
        g, Z = t.grad(theta, 1.0)
    assert Z == pytest.approx(ref["Z"], rel=1e-12)
    assert rel(g, ref["g"]) < FP64_TOL
    assert maxrel(g, ref["g"]) < FP64_TOL


@pytest.mark.parametrize("name", ["mixture", "mixture_init", "ragged", "tree_small", "mnist_small"])
@pytest.mark.parametrize("theta", [0.5, 0.8])
def test_bh_fp32_mixed(name, theta):
    w, y = workload(name)
    ref = oracle.bh_grad(y, w.indptr, w.indices, w.values, theta=theta, exag=1.0)
    with make("fp32", w, y) as t:
        g, Z = t.grad(theta, 1.0)
    assert Z == pytest.approx(ref["Z"], rel=1e-4)
    assert rel(g, ref["g"]) < FP32_TOL
    assert worst_row(g, ref) < FP32_ROW_TOL


@pytest.mark.parametrize("name", ["mixture", "ragged"])
def test_exact_fp32_mixed(name):
    w, y = workload(name)
    ref = oracle.exact_grad(y, w.indptr, w.indices, w.values, exag=12.0)
    with make("fp32", w, y) as t:
        g, Z = t.grad(0.0, 12.0)
    assert Z == pytest.approx(ref["Z"], rel=1e-5)
    assert rel(g, ref["g"]) < FP32_TOL
    assert worst_row(g, ref, 12.0) < FP32_ROW_TOL


@pytest.mark.parametrize("theta", [0.0, 0.5])
def test_steps_fp64_track_oracle(theta):
    w, y = workload("mixture")
    lr = w.n / 12000.0
    yo, vo, _ = oracle.step(y, np.zeros_like(y), w.indptr, w.indices, w.values, 10, theta, 12.0, lr, 0.5)
    with make("fp64", w, y) as t:
        t.step(10, theta, 12.0, lr, 0.5)
        yg = t.get_Y()
        vg, _, it = t.get_state()
    assert it == 10
    assert rel(yg, yo) < FP64_TOL
    assert rel(vg, vo) < 1e-8


def test_steps_with_gains_and_metric2():
    w, y = workload("mixture_init")
    gains = np.ones_like(y)
    yo, vo, go = oracle.step(y, np.zeros_like(y), w.indptr, w.indices, w.values, 5, 0.5, 12.0, 1.0, 0.5,
                             gains=gains, metric_pow=2)
    with make("fp64", w, y, use_gains=True, metric_pow=2) as t:
        t.step(5, 0.5, 12.0, 1.0, 0.5)
        yg = t.get_Y()
        vg, gg, _ = t.get_state()
    assert rel(yg, yo) < FP64_TOL
    assert np.array_equal(gg, go)


@pytest.mark.parametrize("theta", [0.0, 0.5])
def test_kl(theta):
    w, y = workload("mixture")
    ref = oracle.kl(y, w.indptr, w.indices, w.values, theta=theta)
    with make("fp64", w, y) as t:
        assert t.kl(theta) == pytest.approx(ref, rel=1e-10)
    with make("fp32", w, y) as t:
        assert t.kl(theta) == pytest.approx(ref, rel=1e-4)


# ---------------------------------------------------------------------------
# Equal-area radial splits (Eq. EqualAreaSplitting): gradient, Z and steps
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["mixture", "ragged", "tree_small"])
@pytest.mark.parametrize("theta", [0.2, 0.5, 0.8])
def test_bh_fp64_equal_area(name, theta):
    w, y = workload(name)
    ref = oracle.bh_grad(y, w.indptr, w.indices, w.values, theta=theta, exag=1.0, split_rule=1)
    with make("fp64", w, y, split_rule="equal_area") as t:
        g, Z = t.grad(theta, 1.0)
    assert Z == pytest.approx(ref["Z"], rel=1e-12)
    assert rel(g, ref["g"]) < FP64_TOL
    assert maxrel(g, ref["g"]) < FP64_TOL


@pytest.mark.parametrize("name", ["mixture", "mixture_init", "ragged", "tree_small", "mnist_small"])
@pytest.mark.parametrize("theta", [0.5, 0.8])
def test_bh_fp32_mixed_equal_area(name, theta):
    w, y = workload(name)
    ref = oracle.bh_grad(y, w.indptr, w.indices, w.values, theta=theta, exag=1.0, split_rule=1)
    with make("fp32", w, y, split_rule="equal_area") as t:
        g, Z = t.grad(theta, 1.0)
    assert Z == pytest.approx(ref["Z"], rel=1e-4)
    assert rel(g, ref["g"]) < FP32_TOL
    assert worst_row(g, ref) < FP32_ROW_TOL


def test_steps_fp64_equal_area_track_oracle():
    w, y = workload("mixture")
    lr = w.n / 12000.0
    yo, vo, _ = oracle.step(y, np.zeros_like(y), w.indptr, w.indices, w.values, 10, 0.5, 12.0, lr, 0.5,
                            split_rule=1)
    with make("fp64", w, y, split_rule="equal_area") as t:
        t.step(10, 0.5, 12.0, lr, 0.5)
        yg = t.get_Y()
        vg, _, it = t.get_state()
    assert it == 10
    assert rel(yg, yo) < FP64_TOL
    assert rel(vg, vo) < 1e-8


def test_kl_equal_area():
    w, y = workload("mixture")
    ref = oracle.kl(y, w.indptr, w.indices, w.values, theta=0.5, split_rule=1)
    with make("fp64", w, y, split_rule="equal_area") as t:
        assert t.kl(0.5) == pytest.approx(ref, rel=1e-10)


def test_paper_printed_gradient_form():
    w, y = workload("mixture")
    ref = oracle.bh_grad(y, w.indptr, w.indices, w.values, theta=0.5, grad_form=1)
    with make("fp64", w, y, grad_form="paper") as t:
        g, _ = t.grad(0.5, 1.0)
    assert rel(g, ref["g"]) < FP64_TOL


# ---------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------

def tiny_csr(n, seed=0):
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for i in range(n):
        for j in rng.choice(n, size=min(3, n - 1), replace=False):
            if j != i:
                rows += [i, j]
                cols += [j, i]
    P = np.zeros((n, n))
    P[rows, cols] = 1.0
    P /= max(P.sum(), 1)
    indptr = np.zeros(n + 1, np.int64)
    indices, values = [], []
    for i in range(n):
        nz = np.nonzero(P[i])[0]
        indices += nz.tolist()
        values += P[i, nz].tolist()
        indptr[i + 1] = len(indices)
    return indptr, np.array(indices, np.int32), np.array(values)


@pytest.mark.parametrize("case", ["one", "two", "dups", "origin", "rim", "n33"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_degenerate_inputs(case, prec):
    rng = np.random.default_rng(9)
    if case == "one":
        y = np.array([[0.3, -0.2]])
    elif case == "two":
        y = np.array([[0.3, -0.2], [-0.1, 0.5]])
    elif case == "dups":
        base = rng.normal(0, 0.2, (40, 2))
        y = np.concatenate([base, base[:15], base[:3]])
    elif case == "origin":
        y = np.zeros((37, 2))
    elif case == "rim":
        phi = rng.uniform(0, 2 * np.pi, 300)
        r = 1 - 10 ** rng.uniform(-7, -2, 300)
        y = np.stack([r * np.cos(phi), r * np.sin(phi)], 1)
    else:
        y = rng.normal(0, 0.3, (33, 2))
    n = y.shape[0]
    ip, ix, vv = tiny_csr(n) if n > 1 else (np.zeros(2, np.int64), np.zeros(0, np.int32), np.zeros(0))
    tol = FP64_TOL if prec == "fp64" else FP32_TOL
    for theta in (0.0, 0.5):
        ref = oracle.bh_grad(y, ip, ix, vv, theta=theta)
        t = HyperbolicTSNE(precision=prec)
        t.set_P(ip, ix, vv)
        t.set_Y(y)
        g, Z = t.grad(theta, 1.0)
        assert np.all(np.isfinite(g))
        if n == 1:
            assert Z == 0 and np.all(g == 0)
            continue
        assert Z == pytest.approx(ref["Z"], rel=tol)
        # compare against the size of the two force terms: g itself can vanish
        # (two points with p = q balance exactly)
        scale = 4 * (np.linalg.norm(ref["fattr"]) + np.linalg.norm(ref["frep"]) / ref["Z"])
        assert np.linalg.norm(g - ref["g"]) <= tol * scale
        t.step(3, theta, 1.0, 0.1, 0.5)
        yy = t.get_Y()
        assert np.all(np.linalg.norm(yy, axis=1) < 1)
        t.close()


def test_update_Y_keeps_optimiser_state():
    w, y = workload("mixture")
    lr = w.n / 12000.0
    with make("fp64", w, y) as t:
        t.step(3, 0.5, 12.0, lr, 0.5)
        t.step(2, 0.5, 12.0, lr, 0.5)
        yb = t.get_Y()
    with make("fp64", w, y) as u:
        u.step(3, 0.5, 12.0, lr, 0.5)
        u.update_Y(u.get_Y())                    # same positions: the run continues unchanged
        u.step(2, 0.5, 12.0, lr, 0.5)
        assert np.array_equal(u.get_Y(), yb)
        _, _, it = u.get_state()
        assert it == 5
        from paper_2401_13708_gb300 import HtsError
        with pytest.raises(HtsError, match="EDOMAIN"):
            u.update_Y(np.full((w.n, 2), 0.8))   # |y| > 1


def test_input_validation():
    from paper_2401_13708_gb300 import HtsError
    t = HyperbolicTSNE(precision="fp64")
    with pytest.raises(HtsError, match="ENOTSET"):
        t.step(1, 0.5, 1.0, 1.0, 0.5)
    with pytest.raises(HtsError, match="EDOMAIN"):
        t.set_Y(np.array([[0.5, 0.0], [1.0, 0.0]]))
    bad = (np.array([0, 1, 2], np.int64), np.array([0, 0], np.int32), np.array([0.5, 0.5]))
    with pytest.raises(HtsError, match="ESHAPE"):
        t.set_P(*bad)  # diagonal entry
    ok = (np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32), np.array([0.5, 0.5]))
    t.set_P(*ok)
    with pytest.raises(HtsError, match="ESHAPE"):
        t.set_Y(np.zeros((3, 2)))
    t.set_Y(np.array([[0.1, 0.0], [-0.1, 0.0]]))
    with pytest.raises(HtsError, match="EINVAL"):
        t.step(1, 1.5, 1.0, 1.0, 0.5)
    t.step(2, 0.5, 1.0, 1.0, 0.5)
    # device inputs are validated on the device
    import torch
    dev = (torch.tensor([0, 1, 2], dtype=torch.int64, device="cuda"),
           torch.tensor([1, 5], dtype=torch.int32, device="cuda"),
           torch.tensor([0.5, 0.5], dtype=torch.float64, device="cuda"))
    with pytest.raises(HtsError, match="ESHAPE"):
        t.set_P(*dev)
    # optimiser state: a bad memory kind, a negative count, a host pointer given as device memory
    import ctypes as C
    t.set_P(*ok)
    v = np.zeros((2, 2))
    vp = v.ctypes.data_as(C.c_void_p)
    assert t._lib.hts_set_state(t._ctx, vp, None, 0, 7) == -1          # HTS_EINVAL
    assert t._lib.hts_set_state(t._ctx, vp, None, -1, 0) == -1
    assert t._lib.hts_get_state(t._ctx, vp, None, None, 1) == -1       # host array as HTS_DEVICE
    t.set_state(np.full((2, 2), 1e-3), None, 5)
    assert t.get_state()[2] == 5
    t.close()


def test_device_inputs_and_outputs():
    import torch
    w, y = workload("ragged")
    ref = oracle.bh_grad(y, w.indptr, w.indices, w.values, theta=0.5, exag=1.0)
    t = HyperbolicTSNE(precision="fp64")
    t.set_P(torch.from_numpy(w.indptr).cuda(), torch.from_numpy(w.indices).cuda(),
            torch.from_numpy(w.values).cuda())
    t.set_Y(torch.from_numpy(y).cuda())
    g = torch.empty((w.n, 2), dtype=torch.float64, device="cuda")
    t.grad(0.5, 1.0, out=g)
    torch.cuda.synchronize()
    assert rel(g.cpu().numpy(), ref["g"]) < FP64_TOL
    t.close()
