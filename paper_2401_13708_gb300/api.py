"""Python binding of libhts: argument marshalling only.

Every computation runs in the CUDA library; this module turns numpy arrays
(host memory) and torch CUDA tensors (device memory) into pointers and
checks return codes.  Method names follow the C ABI (hts_set_P ->
HyperbolicTSNE.set_P, ...).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (DEVICE, EQUAL_AREA, EQUAL_LENGTH, EXACT_KL, F32, F64, FP32_MIXED, FP64, HOST, PAPER_EQ, HtsConfig,
                   HtsError, check, load)

_PREC = {"fp64": FP64, "fp32": FP32_MIXED, "fp32_mixed": FP32_MIXED, FP64: FP64, FP32_MIXED: FP32_MIXED}
_SPLIT = {"equal_length": EQUAL_LENGTH, "equal_area": EQUAL_AREA, EQUAL_LENGTH: EQUAL_LENGTH,
          EQUAL_AREA: EQUAL_AREA}
_GRAD = {"exact": EXACT_KL, "exact_kl": EXACT_KL, "paper": PAPER_EQ, "paper_eq": PAPER_EQ, EXACT_KL: EXACT_KL,
         PAPER_EQ: PAPER_EQ}


def _is_torch(x):
    try:
        import torch
        return isinstance(x, torch.Tensor)
    except ImportError:  # pragma: no cover
        return False


def _arg(x, dtype):
    """(pointer, where, keepalive) for a numpy array or a torch tensor."""
    if _is_torch(x):
        import torch
        tdt = {np.float64: torch.float64, np.float32: torch.float32, np.int64: torch.int64,
               np.int32: torch.int32, np.uint64: torch.uint64}[dtype]
        if x.dtype != tdt:
            raise TypeError(f"expected a {tdt} tensor, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if x.is_cuda:
            return C.c_void_p(x.data_ptr()), DEVICE, x
        x = x.numpy()
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data_as(C.c_void_p), HOST, a


class HyperbolicTSNE:
    """One embedding problem on one GPU (an hts_ctx)."""

    def __init__(self, precision="fp32", split_rule="equal_length", grad_form="exact", metric_pow: int = 1,
                 eps: float = 1e-5, use_gains: bool = False, device: int = 0, stream=None):
        self._lib = load()
        cfg = HtsConfig()
        self._lib.hts_default_config(C.byref(cfg))
        cfg.precision = _PREC[precision]
        cfg.split_rule = _SPLIT[split_rule]
        cfg.grad_form = _GRAD[grad_form]
        cfg.metric_pow = int(metric_pow)
        cfg.eps = float(eps)
        cfg.use_gains = int(bool(use_gains))
        cfg.device = int(device)
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device).cuda_stream
            except Exception:  # pragma: no cover
                stream = None
        cfg.stream = C.c_void_p(int(stream) if stream else 0)
        self.config = cfg
        self._ctx = C.c_void_p()
        code = self._lib.hts_create(C.byref(self._ctx), C.byref(cfg))
        if code != 0:
            raise HtsError(code, "hts_create failed")
        self.n = 0

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            self._lib.hts_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, code):
        return check(self._lib, self._ctx, code)

    # -- inputs -------------------------------------------------------------
    def set_P(self, indptr, indices, values):
        """Copy the CSR affinity matrix (int64 indptr, int32 indices, f32/f64 values)."""
        n = int(indptr.shape[0]) - 1
        nnz = int(indices.shape[0])
        vdt = np.float64 if str(values.dtype).endswith("float64") else np.float32
        p0, w0, k0 = _arg(indptr, np.int64)
        p1, w1, k1 = _arg(indices, np.int32)
        p2, w2, k2 = _arg(values, vdt)
        if len({w0, w1, w2}) != 1:
            raise ValueError("indptr, indices and values must all be host or all device")
        self._check(self._lib.hts_set_P(self._ctx, n, nnz, p0, p1, p2, F64 if vdt is np.float64 else F32, w0))
        if n != getattr(self, "n", n):
            self.nseg = 1
        del k0, k1, k2

    def set_Y(self, y):
        """Copy the embedding (n x 2 float64); resets velocity and gains."""
        n = int(y.shape[0])
        p, w, keep = _arg(y, np.float64)
        self._check(self._lib.hts_set_Y(self._ctx, n, p, w))
        if n != getattr(self, "n", n):
            self.nseg = 1  # the library drops segments when n changes
        self.n = n
        del keep

    def update_Y(self, y):
        """Overwrite the positions (same n) and keep velocity, gains and the
        iteration count."""
        if int(y.shape[0]) != self.n:
            raise ValueError("update_Y keeps n; use set_Y for another size")
        p, w, keep = _arg(y, np.float64)
        self._check(self._lib.hts_update_Y(self._ctx, p, w))
        del keep

    def set_cosne(self, lambda1: float = 1.0, lambda2: float = 0.0, x_sqnorm=None):
        """CO-SNE term (|x_i|^2 per point); x_sqnorm=None switches it off."""
        if x_sqnorm is None:
            self._check(self._lib.hts_set_cosne(self._ctx, 1.0, 0.0, None, HOST))
            return
        p, w, keep = _arg(x_sqnorm, np.float64)
        self._check(self._lib.hts_set_cosne(self._ctx, float(lambda1), float(lambda2), p, w))
        del keep

    # -- iteration ----------------------------------------------------------
    def step(self, n_iter: int, theta: float, exaggeration: float, lr: float, momentum: float):
        self._check(self._lib.hts_step(self._ctx, int(n_iter), float(theta), float(exaggeration), float(lr),
                                       float(momentum)))

    def get_Y(self, out=None):
        if out is None:
            out = np.empty((self.n, 2), dtype=np.float64)
        p, w, keep = _arg(out, np.float64)
        self._check(self._lib.hts_get_Y(self._ctx, p, w))
        return out if not isinstance(keep, np.ndarray) or keep is out else keep

    def grad(self, theta: float, exaggeration: float = 1.0, out=None):
        """(g, Z): the Euclidean KL gradient (n x 2) and the normalisation."""
        if out is None:
            out = np.empty((self.n, 2), dtype=np.float64)
        p, w, keep = _arg(out, np.float64)
        z = C.c_double(0.0)
        self._check(self._lib.hts_grad(self._ctx, float(theta), float(exaggeration), p, C.byref(z), w))
        g = out if not isinstance(keep, np.ndarray) or keep is out else keep
        return g, z.value

    def kl(self, theta: float) -> float:
        v = C.c_double(0.0)
        self._check(self._lib.hts_kl(self._ctx, float(theta), C.byref(v)))
        return v.value

    # -- batched embeddings ---------------------------------------------------
    def set_segments(self, offsets, lr_scale=None):
        """Split the n points into independent embeddings [offsets[s], offsets[s+1])."""
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        nseg = off.size - 1
        self.nseg = max(nseg, 1)
        lr = None if lr_scale is None else np.ascontiguousarray(lr_scale, dtype=np.float64)
        if lr is not None and lr.size != nseg:
            raise ValueError("lr_scale needs one value per segment")
        code = self._lib.hts_set_segments(self._ctx, int(nseg), off.ctypes.data_as(C.c_void_p),
                                          None if lr is None else lr.ctypes.data_as(C.c_void_p))
        if code != 0:
            self.nseg = 1  # an error leaves one segment
        self._check(code)

    def segment_Z(self):
        z = np.zeros(getattr(self, "nseg", 1))
        self._check(self._lib.hts_get_segment_Z(self._ctx, z.ctypes.data_as(C.c_void_p)))
        return z

    def kl_segments(self, theta: float):
        v = np.zeros(getattr(self, "nseg", 1))
        self._check(self._lib.hts_kl_segments(self._ctx, float(theta), v.ctypes.data_as(C.c_void_p)))
        return v

    # -- launch shapes --------------------------------------------------------
    def autotune(self, theta: float = 0.5, reps: int = 5):
        """Time the launch-shape candidates on the current problem; returns
        (walk threads per block, attraction lanes per row)."""
        out = (C.c_int * 2)()
        self._check(self._lib.hts_autotune(self._ctx, float(theta), int(reps), out))
        return int(out[0]), int(out[1])

    def set_tuning(self, walk_block: int = 0, attract_lanes: int = 0):
        self._check(self._lib.hts_set_tuning(self._ctx, int(walk_block), int(attract_lanes)))

    def set_walk_split(self, depth: int = -1):
        """Cut depth (0..3) of the split walk for small problems; -1 chooses by size."""
        self._check(self._lib.hts_set_walk_split(self._ctx, int(depth)))

    def get_walk_split(self) -> int:
        """The split walk's cut depth in use (the automatic choice resolved)."""
        d = C.c_int(0)
        self._check(self._lib.hts_get_walk_split(self._ctx, C.byref(d)))
        return int(d.value)

    def get_tuning(self):
        out = (C.c_int * 2)()
        self._check(self._lib.hts_get_tuning(self._ctx, out))
        return int(out[0]), int(out[1])

    def set_graphs(self, enable: bool = True):
        """Replay each step iteration as one CUDA graph (same results, fewer launches)."""
        self._check(self._lib.hts_set_graphs(self._ctx, 1 if enable else 0))

    # -- inspection -----------------------------------------------------------
    def get_keys(self):
        keys = np.empty(self.n, dtype=np.uint64)
        b = np.zeros(2)
        self._check(self._lib.hts_get_keys(self._ctx, keys.ctypes.data_as(C.c_void_p),
                                           b.ctypes.data_as(C.c_void_p), HOST))
        return keys, b

    def get_tree(self):
        m = C.c_int64(0)
        self._check(self._lib.hts_get_tree(self._ctx, 0, C.byref(m), None, None, None, None, None, None))
        m = int(m.value)
        t = {"depth": np.zeros(m, np.int32), "prefix": np.zeros(m, np.uint64), "count": np.zeros(m, np.int64),
             "first": np.zeros(m, np.int64), "ycell": np.zeros((m, 2)), "rcell": np.zeros(m)}
        mm = C.c_int64(0)
        ptr = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
        self._check(self._lib.hts_get_tree(self._ctx, m, C.byref(mm), ptr(t["depth"]), ptr(t["prefix"]),
                                           ptr(t["count"]), ptr(t["first"]), ptr(t["ycell"]), ptr(t["rcell"])))
        return t

    def set_counters(self, enable: bool = True):
        self._check(self._lib.hts_set_counters(self._ctx, int(bool(enable))))

    def get_counters(self):
        """[accepted cells, leaf pairs, warp node visits, query points] of the
        last counted walk, and [4] the kernels launched so far."""
        out = np.zeros(5, dtype=np.int64)
        self._check(self._lib.hts_get_counters(self._ctx, out.ctypes.data_as(C.c_void_p)))
        return out

    def criterion_count(self) -> int:
        """Acceptance tests made by the counted walks (active lanes at internal
        cells), reset by set_counters(True)."""
        v = C.c_int64(0)
        self._check(self._lib.hts_get_criterion_count(self._ctx, C.byref(v)))
        return int(v.value)

    def set_profiling(self, enable: bool = True, serial: bool = False):
        """Per-phase CUDA-event timing; serial=True runs the attractive sum on
        the main stream so that every phase is timed alone."""
        mode = 0 if not enable else (2 if serial else 1)
        self._check(self._lib.hts_set_profiling(self._ctx, mode))

    PHASES = ("keys", "sort", "tree", "walk", "attract", "update")

    def get_profile(self):
        """({phase: ms summed}, iterations) since the last call."""
        ms = np.zeros(6)
        it = C.c_int64(0)
        self._check(self._lib.hts_get_profile(self._ctx, ms.ctypes.data_as(C.c_void_p), C.byref(it)))
        return dict(zip(self.PHASES, ms.tolist())), int(it.value)

    def get_state(self, vel=None, gains=None, with_gains: bool = True):
        """(velocity, gains, iterations run).  `vel` / `gains` may be output
        arrays (numpy, or torch host or CUDA tensors, n x 2 float64, all in the
        same memory); with_gains=False skips the gains (returned as None)."""
        if vel is None:
            vel = np.empty((self.n, 2))
        if gains is None and with_gains:
            gains = np.empty((self.n, 2))
        pv, wv, kv = _arg(vel, np.float64)
        pg, wg, kg = (None, wv, None) if gains is None else _arg(gains, np.float64)
        if wv != wg:
            raise ValueError("vel and gains must both be host or both device memory")
        it = C.c_int64(0)
        self._check(self._lib.hts_get_state(self._ctx, pv, pg, C.byref(it), wv))
        out_v = vel if not isinstance(kv, np.ndarray) or kv is vel else kv
        out_g = gains if kg is None or not isinstance(kg, np.ndarray) or kg is gains else kg
        return out_v, out_g, int(it.value)

    def set_state(self, vel=None, gains=None, iters: int = 0):
        """Restore velocity and / or gains (None leaves a part unchanged)."""
        pv, wv, kv = (None, None, None) if vel is None else _arg(vel, np.float64)
        pg, wg, kg = (None, None, None) if gains is None else _arg(gains, np.float64)
        if wv is not None and wg is not None and wv != wg:
            raise ValueError("vel and gains must both be host or both device memory")
        where = wv if wv is not None else (wg if wg is not None else HOST)
        self._check(self._lib.hts_set_state(self._ctx, pv, pg, int(iters), where))
        del kv, kg

    def sizes(self):
        n, nnz = C.c_int64(0), C.c_int64(0)
        self._check(self._lib.hts_get_sizes(self._ctx, C.byref(n), C.byref(nnz)))
        return int(n.value), int(nnz.value)


def measure_peaks(device: int = 0):
    """Measured issue rates of this GPU: float32 FMA TFLOP/s, special-function
    rsqrt Tops/s, float64 FMA TFLOP/s (roofline denominators)."""
    lib = load()
    out = np.zeros(3)
    code = lib.hts_measure_peaks(int(device), out.ctypes.data_as(C.c_void_p))
    if code != 0:
        raise HtsError(code, "hts_measure_peaks failed")
    return {"fp32_fma_tflops": float(out[0]), "mufu_rsqrt_tops": float(out[1]), "fp64_fma_tflops": float(out[2])}


__all__ = ["HyperbolicTSNE", "measure_peaks", "HtsError", "FP64", "FP32_MIXED", "EQUAL_LENGTH", "EQUAL_AREA", "EXACT_KL", "PAPER_EQ",
           "_lib"]
