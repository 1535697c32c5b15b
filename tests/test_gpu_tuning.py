"""Launch-shape autotuner: every walk block size gives the same walk, every
attraction lane count stays within float32 summation-order noise, and the
tuned context still meets the parity bars against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2401_13708_gb300 import HtsError, HyperbolicTSNE, inputs

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


_w = {}


def problem():
    if "w" not in _w:
        w = inputs.make_workload("gaussian_mixture", seed=5, n=3001)
        _w["w"] = (w, inputs.spread_embedding(w.labels, 5, rho_hi=9.0))
    return _w["w"]


def ctx(precision):
    w, y = problem()
    t = HyperbolicTSNE(precision=precision)
    t.set_P(w.indptr, w.indices, w.values)
    t.set_Y(y)
    return t


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_walk_block_size_does_not_change_results(precision):
    with ctx(precision) as t:
        assert t.get_tuning() == (256, 8)
        g0, z0 = t.grad(0.5, 1.0)
        for wb in (32, 64, 128):
            t.set_tuning(walk_block=wb)
            g, z = t.grad(0.5, 1.0)
            assert np.array_equal(g, g0) and z == z0, wb


def test_attraction_lanes_change_only_rounding():
    w, y = problem()
    ref = oracle.bh_grad(y, w.indptr, w.indices, w.values, theta=0.5, exag=12.0)
    with ctx("fp32") as t:
        g0, _ = t.grad(0.5, 12.0)
        for lanes in (4, 16, 32):
            t.set_tuning(attract_lanes=lanes)
            g, _ = t.grad(0.5, 12.0)
            assert rel(g, g0) < 1e-6, lanes
            assert rel(g, ref["g"]) < 1e-3


def test_autotune_then_parity():
    w, y = problem()
    ref = oracle.bh_grad(y, w.indptr, w.indices, w.values, theta=0.5, exag=1.0)
    with ctx("fp32") as t:
        assert t.get_walk_split() == 3          # 3001 points: 94 chunks, the deepest cut by default
        wb, lanes = t.autotune(0.5, 3)
        assert wb in (32, 64, 128, 256) and lanes in (4, 8, 16, 32)
        assert t.get_tuning() == (wb, lanes)
        assert 0 <= t.get_walk_split() <= 3     # timed at every depth
        g, Z = t.grad(0.5, 1.0)
        assert rel(g, ref["g"]) < 1e-3
        assert Z == pytest.approx(ref["Z"], rel=1e-4)
        t.set_graphs(True)
        t.step(3, 0.5, 12.0, w.n / 12000.0, 0.5)  # tuned shapes inside a captured iteration


def test_tuning_arguments_checked():
    with ctx("fp32") as t:
        for bad in ((48, 0), (512, 0), (0, 3), (0, 64)):
            with pytest.raises(HtsError):
                t.set_tuning(*bad)
        with pytest.raises(HtsError):
            t.autotune(0.5, 0)
        with pytest.raises(HtsError):
            t.autotune(1.5, 1)
        assert t.get_tuning() == (256, 8)
