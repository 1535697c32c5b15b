"""A bounded device-side wait that runs out is reported, and the context stays usable.

The one-sweep sort passes wait, per tile, for the digit counts of earlier
tiles; every wait gives up after a bounded number of polls, sets a status bit
(HTS_ETIMEOUT) and writes no key out of range.  hts_set_wait_test makes the
first tile of every pass withhold its publication and cuts the poll limit to
a few polls, so the other tiles' waits run out within microseconds: nothing
waits forever and nothing faults.  The failed call must leave Y and the
optimiser state unchanged, and the next call (test mode off) must match the
FP64 oracle from that state.
"""
import numpy as np
import pytest

import oracle
from bars import FP64_TOL, rel
from paper_2401_13708_gb300 import HtsError, HyperbolicTSNE, inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("graphs", [False, True])
def test_lookback_timeout_is_reported_and_the_context_recovers(graphs):
    # 20,000 points: the one-sweep sort (more than 4096 keys), 20 tiles per pass
    w = inputs.make_workload("gaussian_mixture", seed=2, n=20000)
    y = inputs.spread_embedding(w.labels, 2)
    lr = w.n / 12000.0
    with HyperbolicTSNE(precision="fp64") as t:
        t.set_P(w.indptr, w.indices, w.values)
        t.set_Y(y)
        t.set_graphs(graphs)
        t.step(2, 0.5, 12.0, lr, 0.5)  # both sort buffers now hold complete permutations
        y1 = t.get_Y()
        v1, g1, _ = t.get_state()
        t._check(t._lib.hts_set_wait_test(t._ctx, 8))
        with pytest.raises(HtsError, match="ETIMEOUT"):
            t.step(3, 0.5, 12.0, lr, 0.5)
        with pytest.raises(HtsError, match="ETIMEOUT"):
            t.grad(0.5, 1.0)
        assert np.array_equal(t.get_Y(), y1)
        v, g, _ = t.get_state()
        assert np.array_equal(v, v1) and np.array_equal(g, g1)
        t._check(t._lib.hts_set_wait_test(t._ctx, 0))
        t.step(1, 0.5, 12.0, lr, 0.5)
        y2 = t.get_Y()
        gr, Z = t.grad(0.5, 1.0)
    yo, _, _ = oracle.step(y1, v1, w.indptr, w.indices, w.values, 1, 0.5, 12.0, lr, 0.5)
    assert rel(y2, yo) < FP64_TOL
    ref = oracle.bh_grad(y2, w.indptr, w.indices, w.values, theta=0.5, exag=1.0)
    assert Z == pytest.approx(ref["Z"], rel=FP64_TOL)
    # g nearly cancels here (attraction against repulsion): compare against the
    # size of the two force terms, as for the degenerate inputs
    scale = 4 * (np.linalg.norm(ref["fattr"]) + np.linalg.norm(ref["frep"]) / ref["Z"])
    assert np.linalg.norm(gr - ref["g"]) <= FP64_TOL * scale


def test_wait_test_argument_checks():
    with HyperbolicTSNE(precision="fp32") as t:
        assert t._lib.hts_set_wait_test(t._ctx, -1) == -1
        assert t._lib.hts_set_wait_test(t._ctx, 5000) == -1
        assert t._lib.hts_set_wait_test(t._ctx, 0) == 0
