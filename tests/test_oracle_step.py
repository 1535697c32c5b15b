"""Pins of the oracle's Riemannian step (Sec. 4.2 exp map + projection, Sec. 5.1 momentum).

References: the exponential map's closed properties (a step of tangent length
|v| covers hyperbolic distance lambda |v|, and translating the new point back
by (-y) gives tanh(lambda |v| / 2) v / |v|), the momentum recursion with a
zero learning rate, and the projection's radius bound.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2401_13708_gb300 import inputs


def problem(n=300, seed=0):
    w = inputs.make_workload("gaussian_mixture", seed=seed, n=n)
    y = inputs.spread_embedding(w.labels, seed, rho_hi=5.0)
    return w, y


@pytest.mark.parametrize("metric_pow", [1, 2])
def test_first_step_length_and_direction(metric_pow):
    w, y = problem()
    lr = 0.05
    g = oracle.exact_grad(y, w.indptr, w.indices, w.values)["g"]
    y1, v1, _ = oracle.step(y, np.zeros_like(y), w.indptr, w.indices, w.values, 1, 0.0, 1.0, lr, 0.5,
                            metric_pow=metric_pow)
    lam = 2 / (1 - (y * y).sum(1))
    v_expect = -lr * g / lam[:, None] ** metric_pow
    assert np.allclose(v1, v_expect, rtol=1e-14, atol=0)
    for i in range(0, y.shape[0], 7):
        # hyperbolic length of the step = lambda |v|  (= lr |g| for metric_pow 1)
        d = oracle.dist(y[i], y1[i])
        nv = np.linalg.norm(v_expect[i])
        assert d == pytest.approx(lam[i] * nv, rel=1e-7)
        if metric_pow == 1:
            assert d == pytest.approx(lr * np.linalg.norm(g[i]), rel=1e-7)
        back = oracle.mobius_add(-y[i], y1[i])
        assert np.allclose(back, math.tanh(lam[i] * nv / 2) * v_expect[i] / nv, rtol=1e-5, atol=1e-15)


def test_momentum_with_zero_learning_rate():
    w, y = problem(100)
    rng = np.random.default_rng(3)
    v0 = rng.normal(0, 1e-2, y.shape)
    mu = 0.8
    y1, v1, _ = oracle.step(y, v0, w.indptr, w.indices, w.values, 2, 0.0, 1.0, 0.0, mu)
    assert np.allclose(v1, mu * mu * v0, rtol=1e-15)
    for i in range(0, 100, 9):
        mid = oracle.project(oracle.exp_map(y[i], mu * v0[i]))
        end = oracle.project(oracle.exp_map(mid, mu * mu * v0[i]))
        assert np.allclose(y1[i], end, rtol=1e-14, atol=1e-16)


def test_projection_keeps_points_inside():
    w, y = problem(200)
    y = y.copy()
    y[:10] *= (1 - 2e-6) / np.linalg.norm(y[:10], axis=1)[:, None]
    v = 0.5 * y / np.linalg.norm(y, axis=1)[:, None]  # push outwards hard
    y1, _, _ = oracle.step(y, v, w.indptr, w.indices, w.values, 1, 0.5, 1.0, 0.0, 1.0)
    r = np.linalg.norm(y1, axis=1)
    # reading R9: anything that reached 1 - eps/2 is put back at radius 1 - eps
    assert np.all(r < 1 - 0.5e-5)
    assert np.all(r[:10] == pytest.approx(1 - 1e-5, rel=1e-14))


def test_gains_rule():
    # Reading R8: +0.2 where the gradient and the velocity disagree in sign,
    # *0.8 where they agree, floor 0.01.
    w, y = problem(50)
    g = oracle.exact_grad(y, w.indptr, w.indices, w.values)["g"]
    v0 = np.where(np.arange(100).reshape(50, 2) % 3 == 0, 1.0, -1.0) * 1e-3
    gains0 = np.full_like(y, 1.0)
    gains0[0, 0] = 0.011
    _, _, gn = oracle.step(y, v0, w.indptr, w.indices, w.values, 1, 0.0, 1.0, 0.0, 1.0, gains=gains0)
    agree = (g > 0) == (v0 > 0)
    expect = np.where(agree, gains0 * 0.8, gains0 + 0.2)
    expect = np.maximum(expect, 0.01)
    assert np.allclose(gn, expect, rtol=1e-15)


def test_bh_step_tracks_exact_step():
    # theta -> 0 makes the BH step the exact step
    w, y = problem(400)
    v = np.zeros_like(y)
    ye, _, _ = oracle.step(y, v, w.indptr, w.indices, w.values, 3, 0.0, 12.0, 0.1, 0.5)
    yb, _, _ = oracle.step(y, v, w.indptr, w.indices, w.values, 3, 1e-9, 12.0, 0.1, 0.5)
    assert np.allclose(ye, yb, rtol=1e-12, atol=1e-15)
