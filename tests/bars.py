"""Parity bars shared by the GPU tests.

  * HTS_FP64: relative 1e-9 (global L2 and elementwise against the largest
    component).
  * HTS_FP32_MIXED: relative L2 1e-3 over all compared rows, and the same bar
    row by row: for every row i,
        |g^_i - g_i| <= 1e-3 * s_i,   s_i = 4 (exag |F_attr,i| + |F_rep,i| / Z),
    s_i being the size of the two force terms whose difference is g_i
    (Eq. KlGradientHyperbolicSplit).  s_i >= |g_i|; it is the floor a row
    needs where the two terms nearly cancel.
"""
import numpy as np

FP64_TOL = 1e-9
FP32_TOL = 1e-3
FP32_ROW_TOL = 1e-3


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def maxrel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def row_scale(ref, exag=1.0):
    """s_i = 4 (exag |F_attr,i| + |F_rep,i| / Z) for an oracle result dict."""
    fa = np.linalg.norm(np.asarray(ref["fattr"]).reshape(-1, 2), axis=1)
    fr = np.linalg.norm(np.asarray(ref["frep"]).reshape(-1, 2), axis=1)
    z = float(ref["Z"])
    return 4.0 * (exag * fa + (fr / z if z > 0 else 0.0))


def worst_row(g, ref, exag=1.0):
    """max_i |g^_i - g_i| / s_i (0 for an empty set of rows)."""
    d = np.linalg.norm(np.asarray(g).reshape(-1, 2) - np.asarray(ref["g"]).reshape(-1, 2), axis=1)
    if d.size == 0:
        return 0.0
    s = np.maximum(row_scale(ref, exag), np.linalg.norm(np.asarray(ref["g"]).reshape(-1, 2), axis=1))
    s = np.maximum(s, 1e-300)
    return float(np.max(d / s))
