"""FP64 CPU oracle for hyperbolic t-SNE (ctypes wrapper around hts_oracle.c).

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
CPU-baseline / reference arm import this package; the CUDA product path
(``paper_2401_13708_gb300``) never does, and this package never imports it.

Every function takes and returns numpy float64 arrays; y is (n, 2) row-major.
The paper sections and equations each routine follows are cited in
hts_oracle.c.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hts_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libhts_oracle.so")
_lock = threading.Lock()
_lib = None

GRAD_EXACT_KL = 0
GRAD_PAPER_EQ = 1
SPLIT_EQUAL_LENGTH = 0
SPLIT_EQUAL_AREA = 1
LEVELS = 29


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            d, i64, i32, f64p = C.c_double, C.c_int64, C.c_int, C.POINTER(C.c_double)
            vp = C.c_void_p
            sig = {
                "ho_set_threads": (i32, [i32]),
                "ho_lambda": (d, [vp]),
                "ho_acosh1p": (d, [d]),
                "ho_dist": (d, [vp, vp]),
                "ho_dist_grad": (None, [vp, vp, vp]),
                "ho_mobius_add": (None, [vp, vp, vp]),
                "ho_exp_map": (None, [vp, vp, vp]),
                "ho_project": (None, [vp, d, vp]),
                "ho_einstein_midpoint": (None, [i64, vp, vp]),
                "ho_rcell": (d, [d, d, d]),
                "ho_exact_grad": (None, [i64, vp, vp, vp, vp, d, i32, vp, vp, vp, vp, vp]),
                "ho_kl_given_Z": (d, [i64, vp, vp, vp, vp, d]),
                "ho_exact_Z": (d, [i64, vp]),
                "ho_keys": (None, [i64, vp, i32, vp, vp]),
                "ho_tree_export": (i64, [i64, vp, i32, i32, i64, vp, vp, vp, vp, vp, vp, vp, vp]),
                "ho_bh_grad": (None, [i64, vp, vp, vp, vp, d, d, i32, i32, i64, vp, vp, vp, vp, vp,
                                      vp, vp]),
                "ho_bh_rows": (None, [i64, vp, vp, vp, vp, d, d, i32, i32, d, i64, vp, vp, vp]),
                "ho_kl": (d, [i64, vp, vp, vp, vp, d, i32]),
                "ho_bh_prepare": (vp, [i64, vp, i32]),
                "ho_cosne_H": (d, [i64, vp, vp]),
                "ho_cosne_grad": (None, [i64, vp, vp, d, d, vp, vp]),
                "ho_step_cosne": (None, [i64, vp, vp, vp, vp, vp, i32, d, d, d, d, vp, d, d]),
                "ho_bh_release": (None, [vp]),
                "ho_bh_walk_rows": (None, [vp, vp, vp, vp, vp, d, d, i32, d, i64, vp, vp]),
                "ho_step": (None, [i64, vp, vp, vp, vp, vp, vp, i32, d, d, d, d, i32, i32, i32, d,
                                   i32]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            del f64p
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _csr(indptr, indices, values):
    if indptr is None:
        return None, None, None
    return (np.ascontiguousarray(indptr, dtype=np.int64), np.ascontiguousarray(indices, dtype=np.int32),
            _f64(values))


def set_threads(k: int = 0) -> int:
    """Set the OpenMP thread count (k <= 0 keeps it); returns the count in use."""
    return int(_load().ho_set_threads(int(k)))


# -- geometry ---------------------------------------------------------------

def lam(y):
    return _load().ho_lambda(_p(_f64(y)))


def acosh1p(delta: float) -> float:
    return _load().ho_acosh1p(float(delta))


def dist(a, b) -> float:
    return _load().ho_dist(_p(_f64(a)), _p(_f64(b)))


def dist_grad(yi, yj):
    out = np.zeros(2)
    _load().ho_dist_grad(_p(_f64(yi)), _p(_f64(yj)), _p(out))
    return out


def mobius_add(a, b):
    out = np.zeros(2)
    _load().ho_mobius_add(_p(_f64(a)), _p(_f64(b)), _p(out))
    return out


def exp_map(y, v):
    out = np.zeros(2)
    _load().ho_exp_map(_p(_f64(y)), _p(_f64(v)), _p(out))
    return out


def project(y, eps: float = 1e-5):
    out = np.zeros(2)
    _load().ho_project(_p(_f64(y)), float(eps), _p(out))
    return out


def einstein_midpoint(y):
    y = _f64(y).reshape(-1, 2)
    out = np.zeros(2)
    _load().ho_einstein_midpoint(y.shape[0], _p(y), _p(out))
    return out


def rcell(r0: float, r1: float, dphi: float) -> float:
    return _load().ho_rcell(float(r0), float(r1), float(dphi))


# -- exact ------------------------------------------------------------------

def exact_grad(y, indptr=None, indices=None, values=None, exag: float = 1.0, grad_form: int = 0):
    """Exact gradient.  Returns dict g, fattr, frep, zrow, Z."""
    y = _f64(y).reshape(-1, 2)
    n = y.shape[0]
    ip, ix, vv = _csr(indptr, indices, values)
    g, fa, fr, zr = np.zeros((n, 2)), np.zeros((n, 2)), np.zeros((n, 2)), np.zeros(n)
    Z = C.c_double(0.0)
    _load().ho_exact_grad(n, _p(y), _p(ip), _p(ix), _p(vv), float(exag), int(grad_form), _p(g),
                          _p(fa), _p(fr), _p(zr), C.cast(C.pointer(Z), C.c_void_p))
    return {"g": g, "fattr": fa, "frep": fr, "zrow": zr, "Z": Z.value}


def exact_Z(y) -> float:
    y = _f64(y).reshape(-1, 2)
    return _load().ho_exact_Z(y.shape[0], _p(y))


def kl_given_Z(y, indptr, indices, values, Z: float) -> float:
    y = _f64(y).reshape(-1, 2)
    ip, ix, vv = _csr(indptr, indices, values)
    return _load().ho_kl_given_Z(y.shape[0], _p(y), _p(ip), _p(ix), _p(vv), float(Z))


def kl(y, indptr, indices, values, theta: float = 0.0, split_rule: int = 0) -> float:
    y = _f64(y).reshape(-1, 2)
    ip, ix, vv = _csr(indptr, indices, values)
    return _load().ho_kl(y.shape[0], _p(y), _p(ip), _p(ix), _p(vv), float(theta), int(split_rule))


# -- tree -------------------------------------------------------------------

def keys(y, split_rule: int = 0):
    y = _f64(y).reshape(-1, 2)
    out = np.zeros(y.shape[0], dtype=np.uint64)
    b = np.zeros(2)
    _load().ho_keys(y.shape[0], _p(y), int(split_rule), _p(out), _p(b))
    return out, b


def tree_export(y, split_rule: int = 0, which: int = 0):
    """Compressed tree in pre-order (which=0 literal insertion, 1 key-sorted)."""
    y = _f64(y).reshape(-1, 2)
    n = y.shape[0]
    lib = _load()
    m = lib.ho_tree_export(n, _p(y), int(split_rule), int(which), 0, *([None] * 8))
    out = {
        "depth": np.zeros(m, dtype=np.int32), "prefix": np.zeros(m, dtype=np.uint64),
        "count": np.zeros(m, dtype=np.int64), "first": np.zeros(m, dtype=np.int64),
        "ycell": np.zeros((m, 2)), "beta": np.zeros(m), "rcell": np.zeros(m),
        "bounds": np.zeros(2),
    }
    lib.ho_tree_export(n, _p(y), int(split_rule), int(which), m, _p(out["depth"]), _p(out["prefix"]),
                       _p(out["count"]), _p(out["first"]), _p(out["ycell"]), _p(out["beta"]),
                       _p(out["rcell"]), _p(out["bounds"]))
    return out


# -- Barnes-Hut -------------------------------------------------------------

def bh_grad(y, indptr=None, indices=None, values=None, theta: float = 0.5, exag: float = 1.0,
            split_rule: int = 0, grad_form: int = 0, rows=None):
    """BH gradient.  Returns dict g, fattr, frep (for `rows`, default all),
    zall (all n), Z, stats = [accepted cells, leaf pairs, visited nodes]."""
    y = _f64(y).reshape(-1, 2)
    n = y.shape[0]
    ip, ix, vv = _csr(indptr, indices, values)
    r = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    m = n if r is None else r.shape[0]
    g, fa, fr, za = np.zeros((m, 2)), np.zeros((m, 2)), np.zeros((m, 2)), np.zeros(n)
    Z = C.c_double(0.0)
    st = np.zeros(3, dtype=np.int64)
    _load().ho_bh_grad(n, _p(y), _p(ip), _p(ix), _p(vv), float(theta), float(exag), int(split_rule),
                       int(grad_form), m, _p(r), _p(g), _p(fa), _p(fr), _p(za),
                       C.cast(C.pointer(Z), C.c_void_p), _p(st))
    return {"g": g, "fattr": fa, "frep": fr, "zall": za, "Z": Z.value, "stats": st}


def bh_rows(y, indptr, indices, values, theta, exag, Z, rows, split_rule: int = 0, grad_form: int = 0):
    """BH gradient rows with a given Z.  Returns (g [m,2], frep_z [m,3])."""
    y = _f64(y).reshape(-1, 2)
    ip, ix, vv = _csr(indptr, indices, values)
    r = np.ascontiguousarray(rows, dtype=np.int64)
    g = np.zeros((r.shape[0], 2))
    fz = np.zeros((r.shape[0], 3))
    _load().ho_bh_rows(y.shape[0], _p(y), _p(ip), _p(ix), _p(vv), float(theta), float(exag),
                       int(split_rule), int(grad_form), float(Z), r.shape[0], _p(r), _p(g), _p(fz))
    return g, fz


class PreparedTree:
    """Oracle tree built once (literal insertion) for repeated row walks."""

    def __init__(self, y, split_rule: int = 0):
        self.y = _f64(y).reshape(-1, 2)
        self._h = C.c_void_p(_load().ho_bh_prepare(self.y.shape[0], _p(self.y), int(split_rule)))

    def walk_rows(self, rows, indptr=None, indices=None, values=None, theta=0.5, exag=1.0, Z=1.0,
                  grad_form: int = 0):
        ip, ix, vv = _csr(indptr, indices, values)
        r = np.ascontiguousarray(rows, dtype=np.int64)
        g = np.zeros((r.shape[0], 2))
        _load().ho_bh_walk_rows(self._h, _p(self.y), _p(ip), _p(ix), _p(vv), float(theta), float(exag),
                                int(grad_form), float(Z), r.shape[0], _p(r), _p(g))
        return g

    def close(self):
        if self._h:
            _load().ho_bh_release(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def step(y, v, indptr, indices, values, n_iter: int, theta: float, exag: float, lr: float,
         momentum: float, gains=None, split_rule: int = 0, grad_form: int = 0, metric_pow: int = 1,
         eps: float = 1e-5):
    """n_iter Riemannian steps; returns updated copies (y, v, gains)."""
    y = _f64(y).reshape(-1, 2).copy()
    v = _f64(v).reshape(-1, 2).copy()
    use_gains = gains is not None
    gn = _f64(gains).reshape(-1, 2).copy() if use_gains else None
    ip, ix, vv = _csr(indptr, indices, values)
    _load().ho_step(y.shape[0], _p(y), _p(v), _p(gn), _p(ip), _p(ix), _p(vv), int(n_iter),
                    float(theta), float(exag), float(lr), float(momentum), int(split_rule),
                    int(grad_form), int(metric_pow), float(eps), int(use_gains))
    return y, v, gn


# -- CO-SNE objective (Sec. 4.3) ----------------------------------------------

def cosne_H(y, xsq) -> float:
    y = _f64(y).reshape(-1, 2)
    x = _f64(xsq)
    return _load().ho_cosne_H(y.shape[0], _p(y), _p(x))


def cosne_grad(y, xsq, l1, l2, g_kl):
    """lambda1 g_KL - (4 lambda2 / n)(|x|^2 - |y|^2) y."""
    y = _f64(y).reshape(-1, 2)
    x = _f64(xsq)
    gk = _f64(g_kl).reshape(-1, 2)
    out = np.zeros_like(y)
    _load().ho_cosne_grad(y.shape[0], _p(y), _p(x), float(l1), float(l2), _p(gk), _p(out))
    return out


def step_cosne(y, v, indptr, indices, values, n_iter, theta, exag, lr, momentum, xsq, l1, l2):
    y = _f64(y).reshape(-1, 2).copy()
    v = _f64(v).reshape(-1, 2).copy()
    ip, ix, vv = _csr(indptr, indices, values)
    x = _f64(xsq)
    _load().ho_step_cosne(y.shape[0], _p(y), _p(v), _p(ip), _p(ix), _p(vv), int(n_iter), float(theta), float(exag),
                          float(lr), float(momentum), _p(x), float(l1), float(l2))
    return y, v
