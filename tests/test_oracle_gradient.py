"""Pins of the oracle's exact gradient, Z and KL.

Independent references used here:
  * a brute-force KL(P||Q^H) written with torch.acosh over a dense P
    (the plain definition, Eq. KLDivergence with Eq. LowDimensionalProbabilityHyperbolic),
    differentiated by torch autograd and by central finite differences;
  * the Euclidean t-SNE gradient (Eq. KLGradient), which the hyperbolic one
    approaches as the embedding shrinks to the origin: G_H(Y) -> 2 G_E(2Y);
  * the three Killing fields of the disk (rotation and two boosts): the
    exact gradient of any isometry-invariant cost is orthogonal to them.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2401_13708_gb300 import inputs


def small_problem(n=24, seed=0, scale=0.5):
    x, lab = inputs.gaussian_mixture(n, 10, 3, seed)
    ip, ix, vv = inputs.affinities_csr(x, perplexity=5.0, k=10)
    rng = np.random.default_rng(seed + 100)
    r = scale * np.sqrt(rng.random(n))
    phi = rng.uniform(0, 2 * np.pi, n)
    y = np.stack([r * np.cos(phi), r * np.sin(phi)], 1)
    return y, ip, ix, vv


def dense_p(n, ip, ix, vv):
    P = np.zeros((n, n))
    for i in range(n):
        P[i, ix[ip[i]:ip[i + 1]]] = vv[ip[i]:ip[i + 1]]
    return P


def kl_torch(Y, P):
    n = Y.shape[0]
    sq = (Y * Y).sum(1)
    diff = Y[:, None, :] - Y[None, :, :]
    s = (diff * diff).sum(-1)
    eye = torch.eye(n, dtype=torch.bool)
    gam = 1 + 2 * s / ((1 - sq)[:, None] * (1 - sq)[None, :])
    gam = torch.where(eye, torch.full_like(gam, 2.0), gam)
    d = torch.acosh(gam)
    w = torch.where(eye, torch.zeros_like(gam), 1 / (1 + d * d))
    q = w / w.sum()
    Pt = torch.as_tensor(P)
    mask = Pt > 0
    return (Pt[mask] * torch.log(Pt[mask] / q[mask])).sum(), w.sum()


def test_kl_and_Z_against_brute_force():
    y, ip, ix, vv = small_problem()
    n = y.shape[0]
    C, Z = kl_torch(torch.tensor(y), dense_p(n, ip, ix, vv))
    ex = oracle.exact_grad(y, ip, ix, vv)
    assert ex["Z"] == pytest.approx(float(Z), rel=1e-13)
    assert oracle.exact_Z(y) == pytest.approx(float(Z), rel=1e-13)
    assert oracle.kl(y, ip, ix, vv, theta=0.0) == pytest.approx(float(C), rel=1e-11)


@pytest.mark.parametrize("scale", [0.3, 0.9])
def test_exact_gradient_equals_autograd_of_kl(scale):
    y, ip, ix, vv = small_problem(scale=scale)
    n = y.shape[0]
    Y = torch.tensor(y, requires_grad=True)
    C, _ = kl_torch(Y, dense_p(n, ip, ix, vv))
    C.backward()
    g = oracle.exact_grad(y, ip, ix, vv)["g"]
    assert np.allclose(g, Y.grad.numpy(), rtol=1e-9, atol=1e-12 * np.abs(g).max())


def test_exact_gradient_finite_difference():
    # central differences of the oracle's own KL (h = 1e-6, FP64)
    y, ip, ix, vv = small_problem(n=16, seed=3, scale=0.8)
    g = oracle.exact_grad(y, ip, ix, vv)["g"]
    h = 1e-6
    fd = np.zeros_like(y)
    for i in range(y.shape[0]):
        for c in range(2):
            yp, ym = y.copy(), y.copy()
            yp[i, c] += h
            ym[i, c] -= h
            fd[i, c] = (oracle.kl(yp, ip, ix, vv, 0.0) - oracle.kl(ym, ip, ix, vv, 0.0)) / (2 * h)
    assert np.linalg.norm(fd - g) / np.linalg.norm(g) < 1e-6


def test_printed_equation_lacks_distance_factor():
    # Reading R1: the form printed as Eq. KLGradientHyperbolic (without d_ij)
    # is not the derivative of KL; the default form is.
    y, ip, ix, vv = small_problem(scale=0.9)
    n = y.shape[0]
    Y = torch.tensor(y, requires_grad=True)
    C, _ = kl_torch(Y, dense_p(n, ip, ix, vv))
    C.backward()
    ref = Y.grad.numpy()
    printed = oracle.exact_grad(y, ip, ix, vv, grad_form=oracle.GRAD_PAPER_EQ)["g"]
    assert np.linalg.norm(printed - ref) / np.linalg.norm(ref) > 0.1


def euclid_grad(y, P):
    # Eq. KLGradient: 4 sum_j (p_ij - q_ij) (1 + |y_i - y_j|^2)^-1 (y_i - y_j)
    diff = y[:, None, :] - y[None, :, :]
    w = 1 / (1 + (diff ** 2).sum(-1))
    np.fill_diagonal(w, 0)
    q = w / w.sum()
    return 4 * (((P - q) * w)[:, :, None] * diff).sum(1)


def test_euclidean_limit():
    # For |y| -> 0, d^H(y_i, y_j) -> 2 |y_i - y_j|, so the hyperbolic cost is
    # the Euclidean cost at 2Y and G_H(Y) -> 2 G_E(2Y), with O(|y|^2) error.
    y0, ip, ix, vv = small_problem(scale=1.0)
    P = dense_p(y0.shape[0], ip, ix, vv)
    errs = []
    for eps in [1e-2, 1e-3]:
        y = eps * y0
        gh = oracle.exact_grad(y, ip, ix, vv)["g"]
        ge = 2 * euclid_grad(2 * y, P)
        errs.append(np.linalg.norm(gh - ge) / np.linalg.norm(ge))
    assert errs[1] < 1e-5
    assert errs[0] / errs[1] > 50  # quadratic convergence


def test_killing_field_invariants():
    # KL depends on y only through pairwise hyperbolic distances, so its
    # exact gradient is orthogonal to every Killing field of the disk:
    # rotation K(y) = (-y2, y1) and boosts K_a(y) = (1+|y|^2) a - 2 <a,y> y.
    y, ip, ix, vv = small_problem(n=40, seed=7, scale=0.95)
    g = oracle.exact_grad(y, ip, ix, vv, exag=1.0)["g"]
    n2 = (y * y).sum(1)
    rot = -y[:, 1] * g[:, 0] + y[:, 0] * g[:, 1]
    scale = np.abs(g).sum() * np.abs(y).max()
    assert abs(rot.sum()) < 1e-12 * scale
    for a in (np.array([1.0, 0.0]), np.array([0.0, 1.0])):
        K = (1 + n2)[:, None] * a - 2 * (y @ a)[:, None] * y
        terms = (K * g).sum(1)
        assert abs(terms.sum()) < 1e-12 * np.abs(K * g).sum()
    # the invariants hold for the attractive and repulsive parts separately
    ex = oracle.exact_grad(y, ip, ix, vv)
    for part in ("fattr", "frep"):
        f = ex[part]
        assert abs((-y[:, 1] * f[:, 0] + y[:, 0] * f[:, 1]).sum()) < 1e-12 * np.abs(f).sum()


def test_exaggeration_scales_attraction_only():
    y, ip, ix, vv = small_problem()
    a = oracle.exact_grad(y, ip, ix, vv, exag=1.0)
    b = oracle.exact_grad(y, ip, ix, vv, exag=12.0)
    assert np.allclose(b["g"] - a["g"], 4 * 11 * a["fattr"], rtol=1e-12, atol=1e-15)
    assert np.allclose(a["g"], 4 * (a["fattr"] - a["frep"] / a["Z"]), rtol=1e-13, atol=1e-16)


def test_degenerate_inputs():
    # duplicate points: zero force between them, w = 1 in Z; a single point.
    y = np.array([[0.1, 0.2], [0.1, 0.2], [-0.3, 0.05]])
    ex = oracle.exact_grad(y)
    assert np.all(np.isfinite(ex["g"]))
    z01 = 2 * 1.0
    z02 = 1 / (1 + oracle.dist(y[0], y[2]) ** 2)
    assert ex["Z"] == pytest.approx(z01 + 4 * z02, rel=1e-14)
    one = oracle.exact_grad(np.array([[0.2, 0.1]]))
    assert one["Z"] == 0 and np.all(one["g"] == 0)


def test_cosne_gradient_finite_difference():
    # CO-SNE (Sec. 4.3): cost lambda1 KL + (lambda2 / n) sum (|x_i|^2 - |y_i|^2)^2.
    # Central differences of that cost (H by plain numpy) against the oracle's
    # gradient; the printed variation's sign would fail this check.
    y, ip, ix, vv = small_problem(n=14, seed=5, scale=0.7)
    n = y.shape[0]
    xsq = np.random.default_rng(8).uniform(0.0, 0.5, n)
    l1, l2 = 0.7, 3.0

    def cost(yy):
        H = np.mean((xsq - (yy ** 2).sum(1)) ** 2)
        return l1 * oracle.kl(yy, ip, ix, vv, 0.0) + l2 * H

    assert oracle.cosne_H(y, xsq) == pytest.approx(np.mean((xsq - (y ** 2).sum(1)) ** 2), rel=1e-14)
    g = oracle.cosne_grad(y, xsq, l1, l2, oracle.exact_grad(y, ip, ix, vv)["g"])
    h = 1e-6
    fd = np.zeros_like(y)
    for i in range(n):
        for c in range(2):
            yp, ym = y.copy(), y.copy()
            yp[i, c] += h
            ym[i, c] -= h
            fd[i, c] = (cost(yp) - cost(ym)) / (2 * h)
    assert np.linalg.norm(fd - g) / np.linalg.norm(g) < 1e-6
    printed = l1 * oracle.exact_grad(y, ip, ix, vv)["g"] + 4 * l2 / n * (xsq - (y ** 2).sum(1))[:, None] * y
    assert np.linalg.norm(fd - printed) / np.linalg.norm(g) > 1e-2
