"""The allocation-free exact gradient (hts_exact_grad_noalloc).

Some callers cannot allocate device memory -- a plug-in inside a framework or
server whose own allocator owns the device memory budget, or code that cannot
take the device synchronisation of cudaMalloc -- so this entry point keeps its
work arrays in a fixed device array inside the library.  The tests call it
through the C ABI with device buffers (allocated here by the test, not by the
entry point) and check it
  * against the FP64 oracle's exact gradient and Z (relative 1e-9, the float64
    bar of the other parity tests) and against the context API's exact
    gradient (hts_grad at theta = 0), on two calls in a row of different sizes
    (the shared array keeps the previous call's contents);
  * at its capacity, n = HTS_NOALLOC_MAX_N, against hts_grad at theta = 0,
    the oracle on sampled rows (with the oracle's own exact Z), and the
    rotation invariant of the exact gradient;
  * with a point outside the disk (NaN results), and then a valid call again.
The file is collected last, so a failure here leaves every other test run.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from bars import FP64_TOL, maxrel, rel
from paper_2401_13708_gb300 import HyperbolicTSNE, _lib, inputs

pytestmark = pytest.mark.gpu


def _p(t):
    return C.c_void_p(t.data_ptr())


def _call(lib, w, y, exag=12.0):
    """One call on device copies of (w, y); returns (g, Z) on the host."""
    import torch
    dev = torch.device("cuda:0")
    yd = torch.from_numpy(np.ascontiguousarray(y)).to(dev)
    ip = torch.from_numpy(w.indptr).to(dev)
    ix = torch.from_numpy(w.indices).to(dev)
    vv = torch.from_numpy(np.asarray(w.values, np.float64)).to(dev)
    g = torch.full((w.n, 2), 7.0, dtype=torch.float64, device=dev)
    z = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    rc = lib.hts_exact_grad_noalloc(w.n, w.nnz, _p(yd), _p(ip), _p(ix), _p(vv), exag, _lib.EXACT_KL, _p(g),
                                    _p(z), C.c_void_p(stream.cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    return g.cpu().numpy(), float(z.item())


def _context_grad(w, y, exag=12.0):
    with HyperbolicTSNE(precision="fp64") as t:
        t.set_P(w.indptr, w.indices, w.values)
        t.set_Y(y)
        return t.grad(0.0, exag)


def test_noalloc_matches_oracle_and_context_twice():
    import torch
    torch.cuda.set_device(0)
    lib = _lib.load()
    cases = []
    for seed, n in ((0, 2000), (1, 3001)):
        w = inputs.make_workload("gaussian_mixture", seed=seed, n=n)
        y = inputs.spread_embedding(w.labels, seed, rho_hi=8.0)
        ref = oracle.exact_grad(y, w.indptr, w.indices, w.values, exag=12.0)
        cases.append((w, y, ref, _context_grad(w, y)))
    for w, y, ref, (g_ctx, z_ctx) in cases:  # two calls in a row, different sizes
        g, z = _call(lib, w, y)
        assert rel(g, ref["g"]) < FP64_TOL
        assert maxrel(g, ref["g"]) < FP64_TOL
        assert z == pytest.approx(ref["Z"], rel=1e-12)
        assert rel(g, g_ctx) < FP64_TOL
        assert z == pytest.approx(z_ctx, rel=1e-12)


def test_noalloc_at_capacity():
    import torch
    torch.cuda.set_device(0)
    lib = _lib.load()
    n = _lib.NOALLOC_MAX_N
    w = inputs.make_workload("gaussian_mixture", seed=5, n=n, device="cuda")
    y = inputs.spread_embedding(w.labels, 5, rho_hi=8.0)
    g, z = _call(lib, w, y)
    g_ctx, z_ctx = _context_grad(w, y)
    assert rel(g, g_ctx) < FP64_TOL and z == pytest.approx(z_ctx, rel=1e-12)
    # the oracle on sampled rows, including the last point, with its own exact Z
    z_or = oracle.exact_Z(y)
    assert z == pytest.approx(z_or, rel=1e-11)
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([rng.choice(n, 200, replace=False), [0, n - 1]]))
    g_or, _ = oracle.bh_rows(y, w.indptr, w.indices, w.values, 0.0, 12.0, z_or, rows)
    assert rel(g[rows], g_or) < FP64_TOL
    # rotation invariant of the exact gradient: sum_i y_i x g_i = 0
    torque = float(np.sum(y[:, 0] * g[:, 1] - y[:, 1] * g[:, 0]))
    scale = float(np.sum(np.abs(y[:, 0] * g[:, 1]) + np.abs(y[:, 1] * g[:, 0])))
    assert abs(torque) <= 1e-10 * scale


def test_noalloc_point_outside_disk_gives_nan_then_recovers():
    import torch
    torch.cuda.set_device(0)
    lib = _lib.load()
    w = inputs.make_workload("gaussian_mixture", seed=2, n=700)
    y = inputs.spread_embedding(w.labels, 2, rho_hi=6.0)
    bad = y.copy()
    bad[17] = [0.9, 0.6]  # |y| > 1
    g, z = _call(lib, w, bad)
    assert np.all(np.isnan(g)) and np.isnan(z)
    g, z = _call(lib, w, y)  # the flag is cleared by the next call
    ref = oracle.exact_grad(y, w.indptr, w.indices, w.values, exag=12.0)
    assert rel(g, ref["g"]) < FP64_TOL and z == pytest.approx(ref["Z"], rel=1e-12)


def test_noalloc_rejects_sizes_beyond_capacity():
    lib = _lib.load()
    n = _lib.NOALLOC_MAX_N + 1
    dummy = C.c_void_p(1)
    rc = lib.hts_exact_grad_noalloc(n, 0, dummy, dummy, None, None, 1.0, _lib.EXACT_KL, dummy, None, None)
    assert rc == -8  # HTS_ETOOLARGE
