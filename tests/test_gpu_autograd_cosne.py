"""Autograd wrapper of KL and the CO-SNE term against the oracle (GPU).

* KLFunction on a 500-point subset of the hierarchical workload (its own P
  rebuilt on the subset, perplexity 30): backward against torch's central
  finite differences of the forward (h = 1e-6, float64; gradcheck) and
  against the oracle's exact gradient; at theta = 0.5 against the oracle's
  Barnes-Hut gradient.
* CO-SNE: hts_grad / hts_step with |x_i|^2 set, against the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2401_13708_gb300 import HyperbolicTSNE, inputs
from paper_2401_13708_gb300.autograd import kl_divergence

pytestmark = pytest.mark.gpu


def subset_problem(n=500, seed=0):
    x, lab = inputs.binary_tree_diffusion(16, 100, seed)
    rng = np.random.default_rng(seed + 3)
    keep = np.sort(rng.choice(x.shape[0], size=n, replace=False))
    xs = inputs.pca(x[keep], 50)
    ip, ix, vv = inputs.affinities_csr(xs, perplexity=30.0)
    y = inputs.spread_embedding(lab[keep], seed, rho_hi=6.0)
    return xs, ip, ix, vv, y


def test_klfunction_gradcheck_and_oracle():
    xs, ip, ix, vv, y = subset_problem()
    model = HyperbolicTSNE(precision="fp64")
    model.set_P(ip, ix, vv)
    yt = torch.tensor(y, dtype=torch.float64, device="cuda", requires_grad=True)
    loss = kl_divergence(yt, model, 0.0)
    assert float(loss.detach()) == pytest.approx(oracle.kl(y, ip, ix, vv, 0.0), rel=1e-10)
    loss.backward()
    ref = oracle.exact_grad(y, ip, ix, vv)["g"]
    g = yt.grad.cpu().numpy()
    assert np.linalg.norm(g - ref) <= 1e-9 * np.linalg.norm(ref)
    # finite differences of the forward itself (float64, h = 1e-6)
    small = torch.tensor(y[:40], dtype=torch.float64, device="cuda", requires_grad=True)
    # P restricted to the first 40 points, renormalised
    P = np.zeros((40, 40))
    for i in range(40):
        for e in range(ip[i], ip[i + 1]):
            if ix[e] < 40:
                P[i, ix[e]] = vv[e]
    P /= P.sum()
    ip2 = np.zeros(41, np.int64)
    ix2, vv2 = [], []
    for i in range(40):
        nz = np.nonzero(P[i])[0]
        ix2 += nz.tolist()
        vv2 += P[i, nz].tolist()
        ip2[i + 1] = len(ix2)
    m2 = HyperbolicTSNE(precision="fp64")
    m2.set_P(ip2, np.array(ix2, np.int32), np.array(vv2))
    assert torch.autograd.gradcheck(lambda t: kl_divergence(t, m2, 0.0), (small,), eps=1e-6, atol=1e-7,
                                    rtol=1e-5)
    # Barnes-Hut backward = the oracle's BH gradient
    yt.grad = None
    kl_divergence(yt, model, 0.5).backward()
    ref_bh = oracle.bh_grad(y, ip, ix, vv, theta=0.5)["g"]
    assert np.linalg.norm(yt.grad.cpu().numpy() - ref_bh) <= 1e-9 * np.linalg.norm(ref_bh)
    model.close()
    m2.close()


@pytest.mark.parametrize("theta", [0.0, 0.5])
def test_cosne_gradient_and_steps(theta):
    xs, ip, ix, vv, y = subset_problem(n=800, seed=2)
    xsq = (xs ** 2).sum(1)
    xsq = xsq / xsq.max() * 0.8  # scale |x|^2 into the disk's range of |y|^2
    l1, l2 = 1.0, 50.0
    if theta == 0.0:
        gk = oracle.exact_grad(y, ip, ix, vv)["g"]
    else:
        gk = oracle.bh_grad(y, ip, ix, vv, theta=theta)["g"]
    ref = oracle.cosne_grad(y, xsq, l1, l2, gk)
    t = HyperbolicTSNE(precision="fp64")
    t.set_P(ip, ix, vv)
    t.set_Y(y)
    t.set_cosne(l1, l2, xsq)
    g, _ = t.grad(theta, 1.0)
    assert np.linalg.norm(g - ref) <= 1e-9 * np.linalg.norm(ref)
    yo, _ = oracle.step_cosne(y, np.zeros_like(y), ip, ix, vv, 5, theta, 12.0, 0.5, 0.5, xsq, l1, l2)
    t.step(5, theta, 12.0, 0.5, 0.5)
    assert np.linalg.norm(t.get_Y() - yo) <= 1e-9 * np.linalg.norm(yo)
    t.set_cosne(x_sqnorm=None)  # off again: plain KL gradient
    t.set_Y(y)
    g0, _ = t.grad(theta, 1.0)
    assert np.linalg.norm(g0 - gk) <= 1e-9 * np.linalg.norm(gk)
    t.close()
