"""Split walk (several warps per 32-point chunk for small problems): every
cut depth gives each point exactly the interactions of its own walk -- the
accepted-cell and leaf-pair counts do not change -- and the gradient meets
the parity bars against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2401_13708_gb300 import HtsError, HyperbolicTSNE, inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


_cache = {}


def problem(n):
    if n not in _cache:
        w = inputs.make_workload("gaussian_mixture", seed=2, n=n)
        _cache[n] = (w, inputs.spread_embedding(w.labels, 3, rho_hi=9.0))
    return _cache[n]


def run(precision, w, y, theta, depth):
    with HyperbolicTSNE(precision=precision) as t:
        t.set_P(w.indptr, w.indices, w.values)
        t.set_Y(y)
        t.set_walk_split(depth)
        t.set_counters(True)
        g, Z = t.grad(theta, 1.0)
        c = t.get_counters()
    return g, Z, [int(v) for v in c[:2]]


@pytest.mark.parametrize("n", [700, 2000, 4097])
@pytest.mark.parametrize("theta", [0.2, 0.5, 0.8])
def test_split_depths_fp64(n, theta):
    w, y = problem(n)
    ref = oracle.bh_grad(y, w.indptr, w.indices, w.values, theta=theta, exag=1.0)
    g0, Z0, c0 = run("fp64", w, y, theta, 0)
    for depth in (1, 2, 3):
        g, Z, c = run("fp64", w, y, theta, depth)
        assert c == c0, depth                       # the same interactions, each once
        assert rel(g, g0) < 1e-12 and Z == pytest.approx(Z0, rel=1e-13)
        assert rel(g, ref["g"]) < 1e-9 and Z == pytest.approx(ref["Z"], rel=1e-12)


@pytest.mark.parametrize("n", [700, 2000, 4097])
def test_split_depths_fp32(n):
    w, y = problem(n)
    ref = oracle.bh_grad(y, w.indptr, w.indices, w.values, theta=0.5, exag=1.0)
    g0, Z0, c0 = run("fp32", w, y, 0.5, 0)
    for depth in (1, 2, 3):
        g, Z, c = run("fp32", w, y, 0.5, depth)
        assert c == c0, depth
        assert rel(g, g0) < 1e-5
        assert rel(g, ref["g"]) < 1e-3 and Z == pytest.approx(ref["Z"], rel=1e-4)


def test_split_default_and_steps():
    """The default (automatic) depth in a stepping run tracks the oracle."""
    w, y = problem(2000)
    lr = w.n / 12000.0
    yo, _, _ = oracle.step(y, np.zeros_like(y), w.indptr, w.indices, w.values, 2, 0.5, 12.0, lr, 0.5)
    with HyperbolicTSNE(precision="fp64") as t:
        t.set_P(w.indptr, w.indices, w.values)
        t.set_Y(y)
        t.step(2, 0.5, 12.0, lr, 0.5)
        assert rel(t.get_Y(), yo) < 1e-9
        with pytest.raises(HtsError):
            t.set_walk_split(4)
