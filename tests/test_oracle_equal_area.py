"""Pins of the oracle's equal-area radial split (Eq. EqualAreaSplitting, Sec. 4.1).

The oracle splits a cell's radial range at acosh((cosh max + cosh min) / 2)
by working in the coordinate c = cosh(rho) = (1 + |y|^2) / (1 - |y|^2) and
bisecting it (reading R5 with rho^ replaced by c).  None of the references
below calls that arithmetic:

  * radial key bits from a literal bisection in exact rational arithmetic
    (fractions.Fraction): c_j = 1 + 2 |y_j|^2 / (1 - |y_j|^2) (Eq.
    PoincareDistance at the origin) is exact for float64 coordinates, and
    "rho_j >= acosh((cosh a + cosh b) / 2)" is "c_j >= (c_a + c_b) / 2" because
    cosh increases on rho >= 0;
  * cell bounds from the same exact bisection, turned into disk radii through
    rho = 2 asinh(sqrt((c - 1) / 2)), r = tanh(rho / 2); every point lies in its
    cell, and r_cell equals the longest of the cell's diagonal, radial edge
    (rho_1 - rho_0) and outer-arc chord measured between the corners;
  * a pure-Python Barnes-Hut over a literally inserted tree whose nodes carry
    their bounds in rho and split at acosh((cosh a + cosh b) / 2) itself.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from paper_2401_13708_gb300 import inputs

L = oracle.LEVELS


def exact_c(p):
    """cosh of the hyperbolic distance from the origin, exactly (a Fraction)."""
    n2 = Fr(float(p[0])) ** 2 + Fr(float(p[1])) ** 2
    return 1 + 2 * n2 / (1 - n2)


def radial_bits(key):
    q = 0
    for b in range(L):
        q |= ((int(key) >> (2 * b + 1)) & 1) << b
    return q


def angular_bits(key):
    q = 0
    for b in range(L):
        q |= ((int(key) >> (2 * b)) & 1) << b
    return q


def bisect_exact(c, lo, hi, levels=L):
    """Radial cell index of c after `levels` literal equal-area splits of [lo, hi]."""
    q = 0
    for _ in range(levels):
        mid = (lo + hi) / 2
        up = c >= mid
        q = 2 * q + int(up)
        lo, hi = (mid, hi) if up else (lo, mid)
    return q


def rho_of_c(c):
    """Hyperbolic radius acosh(c) for an exact c >= 1, without cancellation."""
    return 2.0 * math.asinh(math.sqrt(float((c - 1) / 2)))


def embeddings():
    rng = np.random.default_rng(5)
    g = rng.normal(0, 0.3, (300, 2))
    g *= np.minimum(1.0, 0.97 / np.linalg.norm(g, axis=1))[:, None]  # inside the disk
    out = {"gauss": g}
    x, lab = inputs.gaussian_mixture(500, 10, 6, 2)
    out["spread"] = inputs.spread_embedding(lab, 4, rho_hi=8.0)
    out["tiny"] = rng.normal(0, 1e-3, (60, 2))
    return out


def c_error_bound(p):
    """Bound on the float64 rounding error of c = (1 + |y|^2) / (1 - |y|^2):
    |y|^2 carries ~1.5 ulp, amplified by dc/d|y|^2 = 2 / (1 - |y|^2)^2, plus
    a few ulp of c itself."""
    eps = np.finfo(np.float64).eps
    n2 = float(p[0]) ** 2 + float(p[1]) ** 2
    c = (1 + n2) / (1 - n2)
    return 8 * eps * c * (1 + 1 / (1 - n2))


@pytest.mark.parametrize("name", ["gauss", "spread", "tiny"])
def test_equal_area_key_bits_from_exact_bisection(name):
    y = embeddings()[name]
    keys, bounds = oracle.keys(y, oracle.SPLIT_EQUAL_AREA)
    cs = [exact_c(p) for p in y]
    lo, hi = min(cs), max(cs)
    jlo, jhi = cs.index(lo), cs.index(hi)
    # root annulus in the split coordinate: [min cosh rho, max cosh rho]
    assert lo >= 1
    assert abs(bounds[0] - float(lo)) <= c_error_bound(y[jlo])
    assert abs(bounds[1] - float(hi)) <= c_error_bound(y[jhi])
    top = (1 << L) - 1
    near = 0
    for j, c in enumerate(cs):
        q = min(bisect_exact(c, lo, hi), top) if hi > lo else 0
        got = radial_bits(keys[j])
        if got != q:
            # allowed only for a point within the rounding of c, c_min and c_max
            # of the split line at the first level where the paths part
            lev = L - (got ^ q).bit_length() + 1
            a, b = lo, hi
            for k in range(lev):
                mid = (a + b) / 2
                if k == lev - 1:
                    break
                a, b = (mid, b) if (q >> (L - 1 - k)) & 1 else (a, mid)
            tol = c_error_bound(y[j]) + c_error_bound(y[jlo]) + c_error_bound(y[jhi])
            assert abs(float(c - mid)) <= tol, (j, lev)
            near += 1
        phi = math.atan2(y[j, 1], y[j, 0]) % (2 * math.pi)
        qb = min(int(math.floor(phi / (2 * math.pi) * (1 << L))), top)
        assert angular_bits(keys[j]) == qb, j
    assert near <= 2


def test_equal_area_differs_from_equal_length():
    y = embeddings()["gauss"]
    k0, _ = oracle.keys(y, oracle.SPLIT_EQUAL_LENGTH)
    k1, _ = oracle.keys(y, oracle.SPLIT_EQUAL_AREA)
    assert np.array_equal(k0 & np.uint64(0x5555555555555555), k1 & np.uint64(0x5555555555555555))  # angles
    assert not np.array_equal(k0, k1)


def parents_of(t):
    par = -np.ones(len(t["depth"]), dtype=np.int64)
    stack = []
    for k in range(len(t["depth"])):
        dk, pk = int(t["depth"][k]), int(t["prefix"][k])
        while stack:
            j = stack[-1]
            dj, pj = int(t["depth"][j]), int(t["prefix"][j])
            if dj < dk and (pk >> (2 * (dk - dj))) == pj:
                break
            stack.pop()
        par[k] = stack[-1] if stack else -1
        stack.append(k)
    return par


def py_dist(a, b):
    s = (a[0] - b[0]) ** 2 + (a[1] - b[1]) ** 2
    return math.acosh(1 + 2 * s / ((1 - a[0] ** 2 - a[1] ** 2) * (1 - b[0] ** 2 - b[1] ** 2)))


@pytest.mark.parametrize("name", ["gauss", "spread"])
def test_equal_area_tree_invariants(name):
    y = embeddings()[name]
    n = y.shape[0]
    t = oracle.tree_export(y, oracle.SPLIT_EQUAL_AREA, 0)
    keys, _ = oracle.keys(y, oracle.SPLIT_EQUAL_AREA)
    cs = [exact_c(p) for p in y]
    lo, hi = min(cs), max(cs)
    par = parents_of(t)
    assert t["count"][0] == n and par[0] == -1 and np.all(par[1:] >= 0)
    internal = t["first"] < 0
    sums = np.zeros_like(t["count"])
    np.add.at(sums, par[1:], t["count"][1:])
    assert np.array_equal(sums[internal], t["count"][internal])
    rho = [rho_of_c(c) for c in cs]
    phi = np.mod(np.arctan2(y[:, 1], y[:, 0]), 2 * np.pi)
    checked = 0
    for k in np.nonzero(internal)[0]:
        dk = int(t["depth"][k])
        if dk == 0 or dk > 10:
            continue
        pk = int(t["prefix"][k])
        ia = sum(((pk >> (2 * q + 1)) & 1) << q for q in range(dk))
        ib = sum(((pk >> (2 * q)) & 1) << q for q in range(dk))
        c0 = lo + (hi - lo) * Fr(ia, 2 ** dk)
        c1 = lo + (hi - lo) * Fr(ia + 1, 2 ** dk)
        rho0, rho1 = rho_of_c(c0), rho_of_c(c1)
        members = [j for j in range(n) if (int(keys[j]) >> (2 * (L - dk))) == pk]
        assert len(members) == t["count"][k]
        for j in members:   # every point inside its cell (exactly, in c)
            assert c0 <= cs[j] <= c1
            assert rho0 - 1e-12 <= rho[j] <= rho1 + 1e-12
        p0, p1 = 2 * math.pi * ib / 2 ** dk, 2 * math.pi * (ib + 1) / 2 ** dk
        assert np.all(phi[members] >= p0 - 1e-12) and np.all(phi[members] <= p1 + 1e-12)
        # r_cell: the longest of diagonal, radial edge and outer-arc chord
        r0, r1 = math.tanh(rho0 / 2), math.tanh(rho1 / 2)
        dp = p1 - p0
        corner_in, corner_out, corner_arc = (r0, 0.0), (r1 * math.cos(dp), r1 * math.sin(dp)), (r1, 0.0)
        want = max(py_dist(corner_in, corner_out), rho1 - rho0, py_dist(corner_arc, corner_out))
        assert t["rcell"][k] == pytest.approx(want, rel=1e-7)
        ym = y[members][:30]
        dmax = max(py_dist(p, q) for p in ym for q in ym)
        assert t["rcell"][k] >= dmax - 1e-9
        checked += 1
    assert checked >= 20


# ---------------------------------------------------------------------------
# Pure-Python Barnes-Hut over a literally inserted tree with explicit bounds
# ---------------------------------------------------------------------------

def literal_bh(y, theta, rule):
    """Repulsive sums F_rep,i and the BH Z (reading R14) over a tree built by
    inserting one point at a time (leaf capacity one, depth cap L).  Each node
    keeps its bounds in the radial variable -- the disk radius r for equal
    length splits, the hyperbolic radius rho for equal-area splits -- and in
    the angle; its children split them at
        r:   (a + b) / 2                          (Eq. EqualEmbeddingLengthsSplitting)
        rho: acosh((cosh a + cosh b) / 2)          (Eq. EqualAreaSplitting)
        phi: (a + b) / 2."""
    n = len(y)
    rad = [math.hypot(*p) for p in y]
    coord = [2 * math.atanh(r) for r in rad] if rule == 1 else rad
    ang = [math.atan2(p[1], p[0]) % (2 * math.pi) for p in y]

    def mid_radial(a, b):
        return math.acosh((math.cosh(a) + math.cosh(b)) / 2) if rule == 1 else (a + b) / 2

    def disk_radius(v):
        return math.tanh(v / 2) if rule == 1 else v

    class Node:
        def __init__(s, depth, a, b, pa, pb):
            s.depth, s.a, s.b, s.pa, s.pb = depth, a, b, pa, pb
            s.kids, s.pts = {}, []

        def child_key(s, j):
            return (int(coord[j] >= mid_radial(s.a, s.b)), int(ang[j] >= (s.pa + s.pb) / 2))

        def make_child(s, key):
            mr, mp = mid_radial(s.a, s.b), (s.pa + s.pb) / 2
            a, b = (mr, s.b) if key[0] else (s.a, mr)
            pa, pb = (mp, s.pb) if key[1] else (s.pa, mp)
            return Node(s.depth + 1, a, b, pa, pb)

    root = Node(0, min(coord), max(coord), 0.0, 2 * math.pi)
    for j in range(n):
        node = root
        while True:
            node.pts.append(j)
            if len(node.pts) == 1 or node.depth == L:
                break  # empty leaf taken, or a bucket at the depth cap
            if not node.kids:  # a leaf with one resident point: push it down
                old = node.pts[0]
                ko = node.child_key(old)
                node.kids[ko] = node.make_child(ko)
                node.kids[ko].pts.append(old)
            k = node.child_key(j)
            if k not in node.kids:
                node.kids[k] = node.make_child(k)
                node.kids[k].pts.append(j)
                break
            node = node.kids[k]

    def midpoint(pts):
        sg = sx = sy = 0.0
        for j in pts:
            n2 = y[j][0] ** 2 + y[j][1] ** 2
            g = (1 + n2) / (1 - n2)
            sg += g
            sx += g * 2 * y[j][0] / (1 + n2)
            sy += g * 2 * y[j][1] / (1 + n2)
        mx, my = sx / sg, sy / sg
        s = math.sqrt(1 - mx * mx - my * my)
        return (mx / (1 + s), my / (1 + s))

    def diameter(node):
        r0, r1 = disk_radius(node.a), disk_radius(node.b)
        dp = node.pb - node.pa
        c = [(r0, 0.0), (r1 * math.cos(dp), r1 * math.sin(dp)), (r1, 0.0)]
        return max(py_dist(c[0], c[1]), py_dist(c[0], c[2]), py_dist(c[2], c[1]))

    def term(yi, yc):
        a = 1 - yi[0] ** 2 - yi[1] ** 2
        b = 1 - yc[0] ** 2 - yc[1] ** 2
        s = (yi[0] - yc[0]) ** 2 + (yi[1] - yc[1]) ** 2
        gam = 1 + 2 * s / (a * b)
        d = math.acosh(gam)
        w = 1 / (1 + d * d)
        if s == 0:
            return w, (0.0, 0.0)
        c = yc[0] ** 2 + yc[1] ** 2 - 2 * (yi[0] * yc[0] + yi[1] * yc[1]) + 1
        den = a * b * math.sqrt(gam * gam - 1)
        dd = (4 * (c * yi[0] / a - yc[0]) / den, 4 * (c * yi[1] / a - yc[1]) / den)
        return w, (w * w * d * dd[0], w * w * d * dd[1])

    F = np.zeros((n, 2))
    Z = 0.0
    accepted = 0

    def walk(node, i):
        nonlocal Z, accepted
        if not node.kids:
            for j in node.pts:
                if j != i:
                    w, f = term(y[i], y[j])
                    Z += w
                    F[i] += f
            return
        if node.depth >= 1:
            yc = midpoint(node.pts)
            d = py_dist(y[i], yc)
            if d > 0 and diameter(node) / d < theta:
                w, f = term(y[i], yc)
                Z += len(node.pts) * w
                F[i] += len(node.pts) * np.array(f)
                accepted += 1
                return
        for key in sorted(node.kids):
            walk(node.kids[key], i)

    for i in range(n):
        walk(root, i)
    return F, Z, accepted


def _points():
    rng = np.random.default_rng(23)
    y = np.concatenate([rng.normal(0, 0.25, (30, 2)), rng.normal([0.7, 0.1], 0.02, (10, 2))])
    assert np.all(np.linalg.norm(y, axis=1) < 0.99)
    return [tuple(p) for p in y], y


@pytest.mark.parametrize("theta", [0.0, 0.3, 0.6, 1.0])
@pytest.mark.parametrize("rule", [0, 1])
def test_bh_matches_literal_python(theta, rule):
    pts, y = _points()
    F, Z, accepted = literal_bh(pts, theta, rule)
    bh = oracle.bh_grad(y, theta=theta, split_rule=rule)
    assert bh["Z"] == pytest.approx(Z, rel=1e-12)
    assert np.allclose(bh["frep"], F, rtol=1e-10, atol=1e-13 * np.abs(F).max())
    assert int(bh["stats"][0]) == accepted
    if theta > 0.5:
        assert accepted > 0


def test_literal_rules_give_different_walks():
    # the two rules build different trees here, so the comparison above checks
    # the equal-area branch itself, not a tree both rules share
    pts, y = _points()
    F0, Z0, a0 = literal_bh(pts, 0.6, 0)
    F1, Z1, a1 = literal_bh(pts, 0.6, 1)
    assert a0 != a1 or not np.allclose(F0, F1, rtol=1e-12, atol=0)
    t0 = oracle.tree_export(y, 0, 0)
    t1 = oracle.tree_export(y, 1, 0)
    assert len(t0["depth"]) != len(t1["depth"]) or not np.array_equal(t0["prefix"], t1["prefix"])
