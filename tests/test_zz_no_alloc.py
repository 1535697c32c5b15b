"""The allocation-free exact gradient (hts_exact_grad_noalloc).

Some callers cannot call cudaMalloc -- work queued during CUDA graph
capture, or plug-ins whose host framework owns the device memory budget --
so this entry point keeps its work arrays in a fixed device array inside the
library.  The test calls it through the C ABI with device buffers (allocated
here by the test, not by the entry point) and checks it against the context
API's exact float64 gradient (hts_grad at theta = 0) within the float64 bar
the other parity tests use, on two calls in a row (the shared array keeps the
first call's contents).  It is collected last so a failure here leaves every
other test already run.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2401_13708_gb300 import HyperbolicTSNE, _lib, inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9


def _p(t):
    return C.c_void_p(t.data_ptr())


def test_noalloc_matches_exact_gradient_twice():
    import torch

    lib = _lib.load()
    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    cases = []
    for seed, n in ((0, 2000), (1, 3001)):
        w = inputs.make_workload("gaussian_mixture", seed=seed, n=n)
        y = inputs.spread_embedding(w.labels, seed, rho_hi=8.0)
        with HyperbolicTSNE(precision="fp64") as t:
            t.set_P(w.indptr, w.indices, w.values)
            t.set_Y(y)
            g_ref, z_ref = t.grad(0.0, 12.0)
        cases.append((w, y, g_ref, z_ref))
    for w, y, g_ref, z_ref in cases:  # two calls in a row, different sizes
        yd = torch.from_numpy(y).to(dev)
        ip = torch.from_numpy(w.indptr).to(dev)
        ix = torch.from_numpy(w.indices).to(dev)
        vv = torch.from_numpy(np.asarray(w.values, np.float64)).to(dev)
        g = torch.full((w.n, 2), float("nan"), dtype=torch.float64, device=dev)
        z = torch.zeros(1, dtype=torch.float64, device=dev)
        rc = lib.hts_exact_grad_noalloc(w.n, w.nnz, _p(yd), _p(ip), _p(ix), _p(vv), 12.0, _lib.EXACT_KL, _p(g),
                                        _p(z), C.c_void_p(stream.cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        gh = g.cpu().numpy()
        assert np.linalg.norm(gh - g_ref) <= FP64_TOL * np.linalg.norm(g_ref)
        assert float(z.item()) == pytest.approx(z_ref, rel=1e-12)


def test_noalloc_rejects_sizes_beyond_capacity():
    lib = _lib.load()
    n = _lib.NOALLOC_MAX_N + 1
    dummy = C.c_void_p(1)
    rc = lib.hts_exact_grad_noalloc(n, 0, dummy, dummy, None, None, 1.0, _lib.EXACT_KL, dummy, None, None)
    assert rc == -8  # HTS_ETOOLARGE
