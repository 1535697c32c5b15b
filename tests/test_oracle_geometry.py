"""Pins of the oracle's Poincare-disk geometry to closed forms and identities.

Every check here is independent of the oracle's own formulas: library
functions (math.atanh, math.tanh, math.acosh), finite differences, group
identities of Moebius addition, and isometry invariance.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def rand_disk(rng, n, rmax=0.95):
    r = rmax * np.sqrt(rng.random(n))
    phi = rng.uniform(0, 2 * np.pi, n)
    return np.stack([r * np.cos(phi), r * np.sin(phi)], 1)


def test_distance_from_origin_closed_form():
    # d(0, y) = 2 atanh |y| (Eq. PoincareDistance with y_i = 0).
    for r in [1e-8, 1e-3, 0.1, 0.5, 0.9, 0.999, 1 - 1e-6]:
        for phi in [0.0, 1.0, 4.0]:
            y = [r * math.cos(phi), r * math.sin(phi)]
            ref = 2 * math.atanh(math.hypot(*y))
            assert oracle.dist([0, 0], y) == pytest.approx(ref, rel=1e-10)


def test_paper_distance_example():
    # The worked value of Sec. 5.1: the closed form is 4 atanh(1 - 1e-4).
    g = GOLDEN["distance_example"]
    d = oracle.dist(g["a"], g["b"])
    assert d == pytest.approx(4 * math.atanh(1 - 1e-4), rel=1e-11)
    assert d == pytest.approx(19.806875102572, rel=1e-11)
    # The printed "approximately 80" is inconsistent with Eq. PoincareDistance.
    assert abs(d - g["paper_printed"]) > 50


def test_distance_symmetry_triangle_and_isometries():
    rng = np.random.default_rng(1)
    y = rand_disk(rng, 60)
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    c = np.array([0.3, -0.45])
    for k in range(0, 57, 3):
        a, b, e = y[k], y[k + 1], y[k + 2]
        dab = oracle.dist(a, b)
        assert dab == pytest.approx(oracle.dist(b, a), rel=1e-13)
        assert dab <= oracle.dist(a, e) + oracle.dist(e, b) + 1e-12
        assert oracle.dist(R @ a, R @ b) == pytest.approx(dab, rel=1e-11)
        # left Moebius translation is an isometry of the disk
        assert oracle.dist(oracle.mobius_add(c, a), oracle.mobius_add(c, b)) == pytest.approx(dab, rel=1e-9)


def test_acosh1p_against_library():
    for delta in [1e-3, 0.1, 1.0, 7.5, 1e3, 1e8]:
        assert oracle.acosh1p(delta) == pytest.approx(math.acosh(1 + delta), rel=1e-13)
    # small delta: acosh(1+x) = sqrt(2x) (1 - x/12 + 3x^2/160 - ...)
    for delta in [1e-16, 1e-12, 1e-8]:
        ser = math.sqrt(2 * delta) * (1 - delta / 12 + 3 * delta ** 2 / 160)
        assert oracle.acosh1p(delta) == pytest.approx(ser, rel=1e-14)


def test_distance_gradient_finite_difference():
    # Eq. PoincareDistanceDerivative against central differences of d.
    rng = np.random.default_rng(2)
    y = rand_disk(rng, 40, 0.9)
    h = 1e-6
    for k in range(0, 40, 2):
        yi, yj = y[k], y[k + 1]
        g = oracle.dist_grad(yi, yj)
        fd = np.zeros(2)
        for c in range(2):
            e = np.zeros(2)
            e[c] = h
            fd[c] = (oracle.dist(yi + e, yj) - oracle.dist(yi - e, yj)) / (2 * h)
        assert np.allclose(g, fd, rtol=1e-6, atol=1e-8)


def test_distance_gradient_accuracy_near_rim():
    # Eq. PoincareDistanceDerivative evaluated literally with 60-digit decimal
    # arithmetic on the same float64 inputs: the oracle must hold 1e-10
    # relative accuracy for close pairs near the boundary of the disk.
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    rng = np.random.default_rng(12)
    worst = 0.0
    for _ in range(200):
        r = 1 - 10 ** rng.uniform(-6, -1.5)
        phi = rng.uniform(0, 2 * np.pi)
        yi = np.array([r * math.cos(phi), r * math.sin(phi)])
        off = 10 ** rng.uniform(-9, -2) * rng.normal(size=2)
        yj = yi + off
        if yj @ yj >= 1:
            yj = yi - off
        a = [Decimal(float(v)) for v in yi]
        b = [Decimal(float(v)) for v in yj]
        al = 1 - a[0] ** 2 - a[1] ** 2
        be = 1 - b[0] ** 2 - b[1] ** 2
        s = (a[0] - b[0]) ** 2 + (a[1] - b[1]) ** 2
        gam = 1 + 2 * s / (al * be)
        c = b[0] ** 2 + b[1] ** 2 - 2 * (a[0] * b[0] + a[1] * b[1]) + 1
        den = al * be * (gam * gam - 1).sqrt()
        ref = np.array([float(4 * (c * a[k] / al - b[k]) / den) for k in range(2)])
        got = oracle.dist_grad(yi, yj)
        worst = max(worst, np.linalg.norm(got - ref) / np.linalg.norm(ref))
        dref = float(((gam + (gam * gam - 1).sqrt())).ln())
        assert oracle.dist(yi, yj) == pytest.approx(dref, rel=1e-10)
    assert worst < 1e-10, worst


def test_mobius_group_identities():
    rng = np.random.default_rng(3)
    y = rand_disk(rng, 20, 0.97)
    for k in range(0, 20, 2):
        a, b = y[k], y[k + 1]
        assert np.allclose(oracle.mobius_add(a, [0, 0]), a, atol=1e-15)
        assert np.allclose(oracle.mobius_add([0, 0], a), a, atol=1e-15)
        assert np.allclose(oracle.mobius_add(-a, a), 0, atol=1e-14)
        # left cancellation (-a) (+) (a (+) b) = b
        assert np.allclose(oracle.mobius_add(-a, oracle.mobius_add(a, b)), b, atol=1e-12)


def test_exp_map_identities():
    rng = np.random.default_rng(4)
    y = rand_disk(rng, 20, 0.9)
    v = rng.normal(0, 0.3, (20, 2))
    for k in range(20):
        assert np.allclose(oracle.exp_map(y[k], [0, 0]), y[k], atol=0)
        # exp_0(v) = tanh(|v|) v / |v|  (lambda_0 = 2)
        nv = np.linalg.norm(v[k])
        assert np.allclose(oracle.exp_map([0, 0], v[k]), math.tanh(nv) * v[k] / nv, atol=1e-15)
        # the step covers hyperbolic distance lambda_y |v|
        z = oracle.exp_map(y[k], v[k])
        lam = 2 / (1 - y[k] @ y[k])
        assert oracle.dist(y[k], z) == pytest.approx(lam * nv, rel=1e-8)
        assert np.linalg.norm(z) < 1
    # conformal factor, Eq. PoincareMetric
    assert oracle.lam([0.6, 0.0]) == pytest.approx(2 / (1 - 0.36), rel=1e-15)


def test_projection_reading():
    eps = 1e-5
    inside = np.array([0.3, -0.4])
    assert np.array_equal(oracle.project(inside, eps), inside)
    for r in [1 - eps / 4, 1.0, 1.2]:
        y = np.array([r * 0.6, r * 0.8])
        p = oracle.project(y, eps)
        assert np.linalg.norm(p) == pytest.approx(1 - eps, rel=1e-15)
        assert np.allclose(p / np.linalg.norm(p), [0.6, 0.8], atol=1e-15)


def test_einstein_midpoint_properties():
    rng = np.random.default_rng(5)
    y = rand_disk(rng, 30, 0.95)
    # a single point is its own midpoint
    assert np.allclose(oracle.einstein_midpoint(y[:1]), y[0], atol=1e-15)
    # y and -y average to the origin
    assert np.allclose(oracle.einstein_midpoint(np.stack([y[1], -y[1]])), 0, atol=1e-15)
    # for two points it is the geodesic midpoint
    for k in range(2, 28, 2):
        a, b = y[k], y[k + 1]
        m = oracle.einstein_midpoint(np.stack([a, b]))
        dab = oracle.dist(a, b)
        assert oracle.dist(a, m) == pytest.approx(dab / 2, rel=1e-8)
        assert oracle.dist(m, b) == pytest.approx(dab / 2, rel=1e-8)
    # rotation equivariance and staying inside the disk
    th = 1.1
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    m = oracle.einstein_midpoint(y)
    assert np.allclose(oracle.einstein_midpoint(y @ R.T), R @ m, atol=1e-13)
    assert np.linalg.norm(m) < 1
    # equivariance under the Moebius isometry x -> c (+) x
    c = np.array([-0.2, 0.35])
    tr = np.stack([oracle.mobius_add(c, p) for p in y[:7]])
    assert np.allclose(oracle.einstein_midpoint(tr), oracle.mobius_add(c, oracle.einstein_midpoint(y[:7])),
                       atol=1e-11)


def _quad_diameter(r0, r1, dphi, m=200):
    """Brute-force longest distance between boundary samples of a polar quad."""
    t = np.linspace(0, 1, m)
    pts = np.concatenate([
        np.stack([r0 * np.cos(dphi * t), r0 * np.sin(dphi * t)], 1),
        np.stack([r1 * np.cos(dphi * t), r1 * np.sin(dphi * t)], 1),
        np.stack([(r0 + (r1 - r0) * t), 0 * t], 1),
        np.stack([(r0 + (r1 - r0) * t) * math.cos(dphi), (r0 + (r1 - r0) * t) * math.sin(dphi)], 1),
    ])
    n2 = (pts ** 2).sum(1)
    s = ((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1)
    gam = 1 + 2 * s / ((1 - n2)[:, None] * (1 - n2)[None, :])
    return float(np.arccosh(gam.max()))


@pytest.mark.parametrize("r0,r1,dphi", [
    (0.0, 0.5, math.pi), (0.1, 0.2, math.pi / 2), (0.5, 0.9, math.pi / 8), (0.9, 0.99, math.pi / 64),
    (0.99, 0.999, 2 * math.pi / 512), (0.3, 0.31, math.pi / 2), (0.0, 0.01, math.pi / 4),
    (0.95, 0.999, math.pi / 4),
])
def test_rcell_is_the_quad_diameter(r0, r1, dphi):
    # Sec. 4.1: the longest internal distance of a polar quad is found among
    # the diagonal, a radial edge and a polar edge.  The oracle's r_cell must
    # equal the brute-force diameter of the quad.
    assert oracle.rcell(r0, r1, dphi) == pytest.approx(_quad_diameter(r0, r1, dphi), rel=1e-6)
