"""Seeded synthetic workloads for hyperbolic t-SNE.

The paper's datasets (Table "Datasets": LUKK, MYELOID8000, PLANARIA, MNIST,
WORDNET, C_ELEGANS) are not available, so these generators produce inputs of
the same shape and structure.  This module is shared by the CUDA path's tests,
the oracle's tests and the benchmark; it holds none of the per-iteration
method (no hyperbolic distance, gradient, tree or update arithmetic).  What it
does compute is the *input* of the method:

* high-dimensional points X (numpy ``default_rng(seed)``, so the bits are the
  same on every platform),
* optional PCA to 50 dimensions (Sec. 5, "Experimental setup": PCA first),
* exact k-nearest neighbours (k = 3 * perplexity, i.e. 90 at perplexity 30),
* the conditional Gaussian affinities of Eq. 1 with sigma_i found by binary
  search on the entropy (perplexity 30 by default),
* the symmetrised, normalised sparse matrix P = (P_cond + P_cond^T) / (2N),
  returned as CSR (int64 indptr, int32 indices, float64 or float32 values),
* an initial embedding Y0 ~ N(0, 1e-4 I) in the Poincare disk, and
* optionally a "spread" embedding that mimics a mid-optimisation state
  (clusters spread over the disk, some points within 1e-4 of the boundary).

Reading of Eq. 1 (garbled in the paper: the numerator divides by 2 sigma_i,
the denominator by 2 sigma_i^2, and (p_j|i + p_i|j)/2 does not sum to one):
p_j|i is proportional to exp(-||x_i - x_j||^2 * beta_i) over the k nearest
neighbours, beta_i chosen so that the entropy equals log(perplexity), and
p_ij = (p_j|i + p_i|j) / (2N), which sums to one.

kNN and the perplexity search run in torch on the requested device, so the
1M-point workload can be prepared on the GPU; everything else is numpy.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

__all__ = [
    "Workload",
    "gaussian_mixture",
    "mnist_like",
    "binary_tree_diffusion",
    "single_cell_like",
    "batched_mixtures",
    "affinities_csr",
    "initial_embedding",
    "spread_embedding",
    "make_workload",
    "make_batched",
    "WORKLOADS",
]


@dataclasses.dataclass
class Workload:
    """One embedding problem: CSR affinities plus an initial embedding."""

    name: str
    n: int
    indptr: np.ndarray  # int64 [n+1]
    indices: np.ndarray  # int32 [nnz]
    values: np.ndarray  # float64 or float32 [nnz]
    y0: np.ndarray  # float64 [n, 2]
    labels: np.ndarray  # int64 [n]
    perplexity: float
    extra: dict = dataclasses.field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.indices.shape[0])


# ---------------------------------------------------------------------------
# High-dimensional point generators (numpy only, platform-independent bits)
# ---------------------------------------------------------------------------

def gaussian_mixture(n: int, d: int = 50, components: int = 10, seed: int = 0,
                     mean_std: float = 2.0):
    """Isotropic Gaussian mixture: means ~ N(0, mean_std^2 I), unit variance."""
    rng = np.random.default_rng(seed)
    means = rng.normal(0.0, mean_std, size=(components, d))
    labels = rng.integers(0, components, size=n)
    x = means[labels] + rng.normal(0.0, 1.0, size=(n, d))
    return x, labels.astype(np.int64)


def mnist_like(n: int = 70000, d: int = 784, classes: int = 10, seed: int = 0,
               keep: float = 0.2, noise: float = 0.1):
    """MNIST-shaped data in [0, 1]^784 with ~80% zeros.

    Point = clip(mask * (template_c + eps), 0, 1) with template_c ~ U(0,1)^d,
    eps ~ N(0, noise^2) and mask ~ Bernoulli(keep) (keep = 0.2: P(zero)=0.8).
    Classes have equal sizes (round robin), shuffled.
    """
    rng = np.random.default_rng(seed)
    templates = rng.uniform(0.0, 1.0, size=(classes, d)).astype(np.float32)
    labels = np.arange(n) % classes
    rng.shuffle(labels)
    x = np.empty((n, d), dtype=np.float32)
    chunk = 8192
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        m = rng.random((e - s, d)) < keep
        eps = rng.normal(0.0, noise, size=(e - s, d))
        x[s:e] = np.clip(m * (templates[labels[s:e]] + eps), 0.0, 1.0)
    return x, labels.astype(np.int64)


def binary_tree_diffusion(depth: int = 16, d: int = 100, seed: int = 0,
                          decay: float = 0.5):
    """Complete binary tree of the given depth (2^(depth+1)-1 nodes).

    Root at the origin of R^d; child = parent + N(0, decay^depth_child I).
    Node order is breadth first (node k has children 2k+1, 2k+2).  The label
    is the depth-3 ancestor (8 classes; shallower nodes get their own index).
    """
    rng = np.random.default_rng(seed)
    n = 2 ** (depth + 1) - 1
    x = np.zeros((n, d), dtype=np.float64)
    node_depth = np.zeros(n, dtype=np.int64)
    for lev in range(1, depth + 1):
        s, e = 2 ** lev - 1, 2 ** (lev + 1) - 1
        idx = np.arange(s, e)
        parent = (idx - 1) // 2
        x[s:e] = x[parent] + rng.normal(0.0, math.sqrt(decay ** lev), size=(e - s, d))
        node_depth[s:e] = lev
    labels = np.arange(n)
    for _ in range(depth):
        deeper = node_depth[labels] > 3
        labels = np.where(deeper, (labels - 1) // 2, labels)
    return x, labels.astype(np.int64)


def single_cell_like(n: int = 1_000_000, d: int = 50, clusters: int = 200,
                     seed: int = 0, sigma: float = 0.5):
    """Single-cell-like log-normal features with Zipf(s=1) cluster sizes.

    mu_c ~ N(0, I_d); x = exp(N(mu_c, sigma^2 I)).  Sizes proportional to 1/rank,
    rounded so they sum to n, assigned in a random permutation.
    """
    rng = np.random.default_rng(seed)
    w = 1.0 / np.arange(1, clusters + 1)
    sizes = np.floor(w / w.sum() * n).astype(np.int64)
    sizes[: n - sizes.sum()] += 1
    labels = np.repeat(np.arange(clusters), sizes)
    rng.shuffle(labels)
    mu = rng.normal(0.0, 1.0, size=(clusters, d)).astype(np.float32)
    x = np.empty((n, d), dtype=np.float32)
    chunk = 1 << 16
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        x[s:e] = np.exp(mu[labels[s:e]] + rng.normal(0.0, sigma, size=(e - s, d)))
    return x, labels.astype(np.int64)


def batched_mixtures(count: int = 64, seed: int = 0, n_lo: int = 500,
                     n_hi: int = 20000, d: int = 50):
    """Parameters of `count` independent mixtures of uneven size.

    N ~ round(exp(U(ln n_lo, ln n_hi))), components ~ U{3..20},
    perplexity ~ U{10, 30, 50}.  Returns a list of (n, components,
    perplexity, sub_seed).
    """
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        comps = int(rng.integers(3, 21))
        perp = float(rng.choice([10.0, 30.0, 50.0]))
        out.append((n, comps, perp, int(rng.integers(0, 2**31 - 1))))
    return out


def pca(x: np.ndarray, k: int = 50, device: str = "cpu") -> np.ndarray:
    """Project centred X onto its top-k principal directions (float64)."""
    import torch

    xt = torch.as_tensor(np.asarray(x), dtype=torch.float64, device=device)
    xt = xt - xt.mean(0, keepdim=True)
    cov = xt.T @ xt
    evals, evecs = torch.linalg.eigh(cov)
    top = evecs[:, torch.argsort(evals, descending=True)[:k]]
    return (xt @ top).cpu().numpy()


# ---------------------------------------------------------------------------
# Affinities: exact kNN + perplexity calibration + symmetrisation (Eq. 1)
# ---------------------------------------------------------------------------

def _knn(x, k: int, device: str):
    """Exact k nearest neighbours (self excluded), squared Euclidean distance."""
    import torch

    on_gpu = device.startswith("cuda")
    dt = torch.float32 if on_gpu else torch.float64
    X = torch.as_tensor(np.asarray(x), dtype=dt, device=device)
    n = X.shape[0]
    sq = (X * X).sum(1)
    chunk = max(1, min(n, (1 << 31) // max(n, 1) if on_gpu else (1 << 25) // max(n, 1)))
    nbr = torch.empty((n, k), dtype=torch.int64, device=device)
    dist = torch.empty((n, k), dtype=torch.float64, device=device)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        dd = sq[s:e, None] + sq[None, :] - 2.0 * (X[s:e] @ X.T)
        dd.clamp_(min=0.0)
        ar = torch.arange(e - s, device=device)
        dd[ar, ar + s] = float("inf")
        v, i = torch.topk(dd, k, dim=1, largest=False, sorted=True)
        nbr[s:e] = i
        # recompute the kept distances in float64 for the perplexity search
        diff = X[s:e, None, :].to(torch.float64) - X[i].to(torch.float64)
        dist[s:e] = (diff * diff).sum(-1)
    return nbr, dist


def _perplexity_search(dist, perplexity: float, tol: float = 1e-5, max_iter: int = 200):
    """Row-wise binary search for beta_i so that entropy(P_i) = log(perplexity)."""
    import torch

    n = dist.shape[0]
    target = math.log(perplexity)
    dmin = dist[:, :1]
    dd = dist - dmin
    beta = torch.ones(n, 1, dtype=torch.float64, device=dist.device)
    lo = torch.zeros_like(beta)
    hi = torch.full_like(beta, float("inf"))
    for _ in range(max_iter):
        p = torch.exp(-dd * beta)
        sp = p.sum(1, keepdim=True)
        h = torch.log(sp) + beta * (p * dd).sum(1, keepdim=True) / sp
        diff = h - target
        if bool((diff.abs() < tol).all()):
            break
        up = diff > 0  # entropy too large: sharpen
        lo = torch.where(up, beta, lo)
        hi = torch.where(up, hi, beta)
        beta = torch.where(up, torch.where(torch.isinf(hi), beta * 2.0, (beta + hi) / 2.0),
                           (beta + lo) / 2.0)
    p = torch.exp(-dd * beta)
    return p / p.sum(1, keepdim=True)


def affinities_csr(x, perplexity: float = 30.0, k: Optional[int] = None,
                   device: str = "cpu", value_dtype=np.float64):
    """Symmetric sparse P in CSR from points X (rows sorted, no diagonal)."""
    import torch

    n = int(np.asarray(x).shape[0])
    if k is None:
        k = int(round(3 * perplexity))
    k = min(k, n - 1)
    nbr, dist = _knn(x, k, device)
    pc = _perplexity_search(dist, perplexity)
    rows = torch.arange(n, device=nbr.device).repeat_interleave(k)
    cols = nbr.reshape(-1)
    vals = pc.reshape(-1)
    idx = torch.stack([torch.cat([rows, cols]), torch.cat([cols, rows])])
    coo = torch.sparse_coo_tensor(idx, torch.cat([vals, vals]) / (2.0 * n), (n, n),
                                  dtype=torch.float64, check_invariants=False).coalesce()
    ij = coo.indices()
    v = coo.values()
    indptr = torch.zeros(n + 1, dtype=torch.int64, device=ij.device)
    indptr[1:] = torch.cumsum(torch.bincount(ij[0], minlength=n), 0)
    return (indptr.cpu().numpy(), ij[1].to(torch.int32).cpu().numpy(),
            v.cpu().numpy().astype(value_dtype))


# ---------------------------------------------------------------------------
# Embeddings
# ---------------------------------------------------------------------------

def initial_embedding(n: int, seed: int = 0, std: float = 1e-2) -> np.ndarray:
    """Y0 ~ N(0, std^2 I) in R^2 (std = 0.01, i.e. variance 1e-4)."""
    rng = np.random.default_rng(seed + 7919)
    return rng.normal(0.0, std, size=(n, 2))


def spread_embedding(labels: np.ndarray, seed: int = 0, max_radius: float = 1 - 1e-4,
                     rho_lo: float = 1.0, rho_hi: float = 12.0, spread: float = 0.6) -> np.ndarray:
    """A synthetic mid-optimisation embedding (polar sampling only).

    Each label c gets a centre at hyperbolic radius rho_c ~ U(rho_lo, rho_hi)
    and angle phi_c ~ U(0, 2 pi); a point of class c is placed at radius
    tanh((rho_c + s * N(0,1)) / 2) and angle phi_c + s * N(0,1) / sinh(rho_c)
    with s = spread, then clipped to max_radius.  This reaches the regime of
    late iterations (points within 1e-4 of the boundary) without running the
    method.
    """
    rng = np.random.default_rng(seed + 104729)
    labels = np.asarray(labels)
    k = int(labels.max()) + 1 if labels.size else 1
    rho_c = rng.uniform(rho_lo, rho_hi, size=k)
    phi_c = rng.uniform(0.0, 2 * math.pi, size=k)
    rho = np.abs(rho_c[labels] + spread * rng.normal(size=labels.shape))
    phi = phi_c[labels] + spread * rng.normal(size=labels.shape) / np.sinh(np.maximum(rho_c[labels], 0.5))
    r = np.minimum(np.tanh(rho / 2.0), max_radius)
    return np.stack([r * np.cos(phi), r * np.sin(phi)], axis=1)


# ---------------------------------------------------------------------------
# The named workloads
# ---------------------------------------------------------------------------

WORKLOADS = {
    "gaussian_mixture": "gaussian-mixture N=2000 D=50 (10 comps), FP64 CSR",
    "mnist_like": "mnist-like N=70000 D=784 -> PCA50, FP32 CSR",
    "binary_tree": "binary-tree diffusion N=131071 D=100 -> PCA50, FP32 CSR",
    "batched_mixtures": "64 batched mixtures N~logU(500,20000)",
    "single_cell": "single-cell-like N=1000000 D=50 (200 Zipf clusters), FP32 CSR",
}


def make_workload(name: str, seed: int = 0, device: str = "cpu", n: Optional[int] = None,
                  perplexity: float = 30.0) -> Workload:
    """Build a named workload (WORKLOADS; the batch has make_batched).  `n`
    overrides the size (tests)."""
    if name == "gaussian_mixture":
        nn = 2000 if n is None else n
        x, lab = gaussian_mixture(nn, 50, 10, seed)
        vdt = np.float64
    elif name == "mnist_like":
        nn = 70000 if n is None else n
        x, lab = mnist_like(nn, 784, 10, seed)
        x = pca(x, 50, device)
        vdt = np.float32
    elif name == "binary_tree":
        if n is None:
            x, lab = binary_tree_diffusion(16, 100, seed)
        else:
            depth = max(1, int(math.floor(math.log2(n + 1))) - 1)
            x, lab = binary_tree_diffusion(depth, 100, seed)
        x = pca(x, 50, device)
        vdt = np.float32
    elif name == "single_cell":
        nn = 1_000_000 if n is None else n
        x, lab = single_cell_like(nn, 50, 200 if nn >= 20000 else 20, seed)
        vdt = np.float32
    else:
        raise ValueError(f"unknown workload {name!r} (the batch is make_batched)")
    indptr, indices, values = affinities_csr(x, perplexity, None, device, vdt)
    nn = int(indptr.shape[0] - 1)
    return Workload(name=WORKLOADS[name], n=nn, indptr=indptr, indices=indices, values=values,
                    y0=initial_embedding(nn, seed), labels=lab, perplexity=perplexity)


def make_batched(count: int = 64, seed: int = 0, device: str = "cpu", n_lo: int = 500, n_hi: int = 20000,
                 d: int = 50, value_dtype=np.float32) -> Workload:
    """`count` independent mixtures as one block-diagonal problem.

    Each embedding s is a Gaussian mixture of n_s points in D=d with its own
    component count and perplexity (batched_mixtures); its P is the usual
    symmetric (P_c + P_c^T) / (2 n_s) over its own points, so every block sums
    to 1.  extra["offsets"] holds the int64 segment boundaries (count + 1),
    extra["params"] the (n, components, perplexity, seed) of each embedding.
    """
    params = batched_mixtures(count, seed, n_lo, n_hi, d)
    ips, ids, vals, ys, labs, offs = [], [], [], [], [], [0]
    for (n, comps, perp, sub) in params:
        x, lab = gaussian_mixture(n, d, comps, sub)
        ip, ix, v = affinities_csr(x, perp, None, device, value_dtype)
        base = offs[-1]
        ips.append(np.asarray(ip, dtype=np.int64))
        ids.append(np.asarray(ix, dtype=np.int64) + base)
        vals.append(np.asarray(v))
        ys.append(initial_embedding(n, sub))
        labs.append(np.asarray(lab))
        offs.append(base + n)
    nnz_base = 0
    indptr_parts = []
    for ip in ips:
        indptr_parts.append(ip[:-1] + nnz_base)
        nnz_base += int(ip[-1])
    indptr = np.concatenate(indptr_parts + [np.array([nnz_base], dtype=np.int64)]).astype(np.int64)
    indices = np.concatenate(ids).astype(np.int32)
    values = np.concatenate(vals).astype(value_dtype)
    nn = offs[-1]
    return Workload(name=f"{count} batched mixtures N~logU({n_lo},{n_hi})", n=nn, indptr=indptr, indices=indices,
                    values=values, y0=np.concatenate(ys), labels=np.concatenate(labs), perplexity=float("nan"),
                    extra={"offsets": np.asarray(offs, dtype=np.int64), "params": params})
