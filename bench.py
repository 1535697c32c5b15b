"""Benchmark: Barnes-Hut hyperbolic t-SNE iterations per second at N = 1M.

Workload: the single-cell-like configuration (N = 1,000,000 points in D = 50,
200 clusters with Zipf sizes, log-normal features, P from exact kNN k = 90 at
perplexity 30, float32 CSR), theta = 0.5, FP32-mixed pair forces.  A step is
one full iteration of the hot path on the device: polar keys, radix sort,
quadtree build, tree walk (repulsion + Z), attractive sum, Z reduction and
the Riemannian update following the paper's protocol (Sec. 5.1): Y0 ~ N(0, 1e-4 I), 250 iterations
with exaggeration 12 and momentum 0.5, then exaggeration 1 and momentum 0.8,
lr = N / 12000.  The warm-up runs the first W iterations of that schedule and
the timed region the next K (default 5 + 995: the paper's 1000 iterations).

Printed (one JSON line on rank 0): iterations/s of the FP32-mixed path, the
all-FP64 GPU path for comparison, the FP32-mixed gradient's relative error
against the FP64 oracle on 10,000 sampled rows, the tree walk's roofline,
the end-to-end rate through the C ABI with host buffers, and the oracle's
own rate on this host's cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BH grad iters/s at N=1M, FP32-mixed vs FP64 GPU, at <=1e-3 grad rel err"
UNIT = "iters/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=995)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--theta", type=float, default=0.5)
    ap.add_argument("--fp64-steps", type=int, default=0, help="0: steps // 20 (at least 3)")
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle error gate / CPU baseline")
    ap.add_argument("--sample-rows", type=int, default=10000)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cache", default="", help="directory to keep the generated workload in (reused if present)")
    ap.add_argument("--shapes", default="",
                    help="walk threads per block,attraction lanes per row (e.g. 256,8) instead of the autotuner")
    ap.add_argument("--suite", action="store_true",
                    help="per-workload report (all five configurations) instead of the headline line")
    ap.add_argument("--workloads", default="gaussian_mixture,mnist_like,binary_tree,batched_mixtures,single_cell",
                    help="workloads of the --suite report")
    ap.add_argument("--split-rule", default="both", choices=["equal_length", "equal_area", "both"],
                    help="--suite: radial split rule(s) of the FP32-mixed runs at theta = 0.5; 'both' also "
                         "reports the per-iteration time gain of equal-length over equal-area splits")
    ap.add_argument("--save-y", default="", help="--profile-only: save Y after the warm-up (.npy)")
    ap.add_argument("--load-y", default="",
                    help="--profile-only: start from this Y (.npy, e.g. from --save-y) instead of running the "
                         "warm-up iterations (a profiler then sees few launches before the timed ones)")
    ap.add_argument("--profile-only", action="store_true",
                    help="FP32-mixed steps only (for a profiler): no FP64 arm, e2e or oracle")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (independent replicas; no data-path collective)
# ---------------------------------------------------------------------------

def dist_setup(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def workload(args, device):
    from paper_2401_13708_gb300 import inputs
    t0 = time.time()
    path = None
    if args.cache:
        os.makedirs(args.cache, exist_ok=True)
        path = os.path.join(args.cache, f"single_cell_n{args.n}_s{args.seed}.npz")
    if path and os.path.exists(path):
        z = np.load(path)
        w = inputs.Workload(name=inputs.WORKLOADS["single_cell"], n=int(z["indptr"].shape[0] - 1), indptr=z["indptr"],
                            indices=z["indices"], values=z["values"], y0=z["y0"], labels=z["labels"],
                            perplexity=30.0)
    else:
        w = inputs.make_workload("single_cell", seed=args.seed, device=device, n=args.n)
        if path:
            np.savez(path, indptr=w.indptr, indices=w.indices, values=w.values, y0=w.y0, labels=w.labels)
    y = inputs.spread_embedding(w.labels, args.seed)  # a harder, rim-heavy state for the error gate
    return w, y, time.time() - t0


def workload_name(n, theta):
    """The headline workload, as both arms name it."""
    return (f"single-cell-like N={n} D=50 (200 Zipf clusters, log-normal), kNN k=90 perplexity 30, FP32 CSR, "
            f"theta={theta}, paper protocol from Y0")


def oracle_pass(w, y, theta, rows):
    """One oracle BH pass: full tree + all n walks (for Z) + gradient rows."""
    import oracle
    cores = oracle.set_threads(0)
    t0 = time.time()
    ref = oracle.bh_grad(y, w.indptr, w.indices, w.values, theta=theta, exag=1.0, rows=rows)
    return ref, time.time() - t0, cores


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    w, _, _ = workload(args, "cuda" if _cuda() else "cpu")
    y = w.y0  # the protocol's start state
    cores = oracle.set_threads(0)
    n = w.n
    rows_per_step = min(n, 2000)
    rng = np.random.default_rng(args.seed + 1)
    ip, ix, vv = (np.ascontiguousarray(w.indptr), np.ascontiguousarray(w.indices),
                  np.ascontiguousarray(w.values, dtype=np.float64))
    t0 = time.time()
    tree = oracle.PreparedTree(y)
    t_tree = time.time() - t0
    times = []
    for s in range(args.warmup + args.steps):
        rows = rng.choice(n, size=rows_per_step, replace=False)
        t0 = time.time()
        tree.walk_rows(rows, ip, ix, vv, args.theta, 1.0, 1.0)
        dt = time.time() - t0
        if s >= args.warmup:
            times.append(dt)
    tree.close()
    t_s = float(np.mean(times))
    t_full = t_tree + (n / rows_per_step) * t_s
    value = 1.0 / t_full
    sample = (f"oracle tree (literal insertion) built once over all {n} points ({t_tree:.2f} s); each timed "
              f"step walks {rows_per_step} random rows (BH repulsion + attraction, {t_s * 1e3:.1f} ms); "
              f"value = 1 / (t_tree + (N / rows) t_step), a full iteration extrapolated from the samples")
    # ms_per_step is the time of one timed (sampled) step, as run; the rate of
    # a full iteration is extrapolated from it (ms_per_iteration)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_s * 1e3,
            "ms_per_iteration": t_full * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(n, args.theta),
                       "n": n, "nnz": w.nnz, "theta": args.theta},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _cuda():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

# Algorithmic FP32 operations of the tree walk (counted from the expressions
# of walk_f32_kernel / pair_terms_f32, an FMA counting 2):
#   criterion test (an open lane at an internal cell): Delta (2), |Delta|^2
#     (3), times 2 il_i (1), compare (1)                             -> 7
#   interaction (accepted cell or leaf pair): Delta, |Delta|^2 and
#     delta = 2 |Delta|^2 il_i il_c (7) + the pair term: clamp (1),
#     delta (delta + 2) (2), sqrt (1), log1p (1), 1 + d^2 (2), rcp (1), w (1),
#     rep (2), coefficient (2), accumulation (4 FMA = 8) (21)       -> 28
# Criterion tests are counted on the device (hts_get_criterion_count), open
# lanes only.
FLOPS_CRITERION = 7
FLOPS_INTERACTION = 28

# Algorithmic DRAM bytes of the memory-bound phases (per point unless noted):
#   keys    Y 16 read + point record 32 + radial 8 written, radial 8 read +
#           key/index 12 written                                        -> 76
#   sort    keys read once for the digit histograms (8) + 8 passes x
#           (12 read + 12 written)                                      -> 200
#   tree    gather 108 (index, Y, record in; sorted record, terms out),
#           radix tree 52, fixed-point scan 168, marks/counts/scan 20,
#           emit 144 (prefix sums in, two 16-byte node records out)       -> ~490
#   attract per non-zero: index 4 + value 4 + the neighbour's position 8
#           (16, counted although the gather is mostly served by L2); per
#           row: indptr 8 + y_i 8 + force 8 (24)
#   update  Y, velocity, both forces 64 read + Z 8 + Y, velocity 32 written -> 104
BYTES_PER_POINT = {"keys": 76, "sort": 200, "tree": 490, "update": 104}
ATTRACT_BYTES_PER_NNZ, ATTRACT_BYTES_PER_ROW = 16, 24


def cpu_model():
    """The host CPU's model name (lscpu or /proc/cpuinfo), for the oracle timing."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def fp64_ops_record():
    """FP64 FLOPs per point of the float64-bound phases, from the committed ncu
    count (profiles/fp64_ops_step_n200k.txt), for each phase whose kernel
    source still hashes as recorded."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "fp64_ops_step_n200k.txt")
    if not os.path.exists(path):
        return {}
    rec = json.load(open(path))
    csrc = os.path.join(ROOT, "paper_2401_13708_gb300", "csrc")
    out = {}
    for ph, flop in rec["fp64_flop_per_point"].items():
        f = rec["phase_source"][ph]
        if hashlib.sha256(open(os.path.join(csrc, f), "rb").read()).hexdigest() == rec["sources_sha256"][f]:
            out[ph] = flop
    return out


def worst_row_err(g, ref, exag=1.0):
    """max over rows of |g^_i - g_i| / (4 (exag |F_attr,i| + |F_rep,i| / Z)): each
    row's error against the size of the two force terms whose difference is g_i."""
    d = np.linalg.norm(np.asarray(g) - ref["g"], axis=1)
    scale = 4.0 * (exag * np.linalg.norm(ref["fattr"], axis=1) + np.linalg.norm(ref["frep"], axis=1) / ref["Z"])
    scale = np.maximum(np.maximum(scale, np.linalg.norm(ref["g"], axis=1)), 1e-300)
    return float(np.max(d / scale)) if d.size else 0.0


EARLY_ITERS = 250  # Sec. 5.2.1: 250 early-exaggeration iterations, then at most 750 plain ones


def protocol(t, it0, k, theta, lr):
    """Iterations it0 .. it0 + k - 1 of the paper's schedule (Sec. 5.1): exaggeration 12
    and momentum 0.5 for the first 250 iterations, then 1 and 0.8; lr = N / 12000."""
    ee = max(0, min(k, EARLY_ITERS - it0))
    if ee:
        t.step(ee, theta, 12.0, lr, 0.5)
    if k - ee:
        t.step(k - ee, theta, 1.0, lr, 0.8)


def run_ours(args, rank, world, local):
    import torch

    from paper_2401_13708_gb300 import HyperbolicTSNE, inputs

    dev = f"cuda:{local}"
    w, y_spread, t_gen = workload(args, dev)
    n = w.n
    y0 = w.y0
    lr = n / 12000.0
    theta = args.theta
    W, K = args.warmup, args.steps
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(local)
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))

    # ---- FP32-mixed: the protocol from Y0 -------------------------------
    t = HyperbolicTSNE(precision="fp32", device=local)
    t.set_P(w.indptr, w.indices, w.values)
    gate_states = {"y0": y0, "spread": y_spread}
    g32 = {}
    for name, ys in gate_states.items():          # gradients for the error gate (no step)
        t.set_Y(ys)
        g32[name] = t.grad(theta, 1.0)
    t.set_Y(y0)
    if args.profile_only and args.load_y:          # a saved state stands in for the warm-up
        t.set_Y(np.load(args.load_y))
    else:
        protocol(t, 0, W, theta, lr)
    if args.profile_only and args.save_y:
        np.save(args.save_y, t.get_Y())
    if args.shapes:                                # fixed launch shapes (e.g. for a profiler run)
        t.set_tuning(*[int(v) for v in args.shapes.split(",")])
        walk_block, attract_lanes = t.get_tuning()
    else:                                          # launch shapes for this problem (Y unchanged)
        walk_block, attract_lanes = t.autotune(theta, 3)
    y_s = t.get_Y()                                # state at the start of the timed segment
    v_s, _, _ = t.get_state()
    if args.profile_only:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        protocol(t, W, K, theta, lr)
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile_only": True, "n": n, "steps": K,
                              "ms_per_step": (time.perf_counter() - t0) * 1e3 / K}), flush=True)
        return
    t.set_profiling(True)
    t.get_profile()
    launches0 = int(t.get_counters()[4])
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        protocol(t, W, K, theta, lr)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    launches = int(t.get_counters()[4]) - launches0
    prof, piters = t.get_profile()
    t.set_profiling(False)
    clocks = clk.summary()
    ms_per_step = ms / K
    value = K * world / (ms / 1e3)
    y_end = t.get_Y()

    # ---- FP32 on the FP64 arm's segment (same start state, same iterations)
    k64 = args.fp64_steps or max(3, K // 20)
    t.set_Y(y_s)
    t.set_state(v_s, None, 0)
    torch.cuda.synchronize()
    e0.record(stream)
    protocol(t, W, k64, theta, lr)
    e1.record(stream)
    torch.cuda.synchronize()
    ms32_seg = max_over_ranks(e0.elapsed_time(e1), world)

    # ---- the timed segment again with the counting walk (deterministic replay)
    t.set_Y(y_s)
    t.set_state(v_s, None, 0)
    t.set_counters(True)
    protocol(t, W, K, theta, lr)
    cnt = t.get_counters()
    crit = t.criterion_count()
    t.set_counters(False)
    acc, pairs, visits, queries = [int(v) for v in cnt[:4]]
    replay_same = bool(np.array_equal(t.get_Y(), y_end))

    # ---- roofline of the dominant kernel (tree walk) --------------------
    walk_ms = prof["walk"] / max(piters, 1)
    flops = ((acc + pairs) * FLOPS_INTERACTION + crit * FLOPS_CRITERION) / K
    sm_mhz = clocks["sm_mhz"] or peaks.get("clocks_under_load", {}).get("sm_mhz_median") or 1462.0
    fp32_peak = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s at the sampled clock
    achieved = flops / (walk_ms * 1e-3) / 1e12
    traffic = None  # DRAM bytes per walk launch from the committed ncu capture, scaled to n
    tf = os.path.join(ROOT, "profiles", "roofline_traffic.txt")
    if os.path.exists(tf):
        import hashlib
        rec = json.load(open(tf))
        src = os.path.join(ROOT, "paper_2401_13708_gb300", "csrc", "traverse.cu")
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        # only counters taken on the kernel as it is now
        if (rec.get("kernel") == "walk_f32_kernel" and rec.get("dram_bytes_per_launch")
                and rec.get("traverse_cu_sha256") == sha):
            traffic = rec["dram_bytes_per_launch"] * n / rec["captured_n"]

    # ---- per-kernel rooflines: the timed segment replayed with every phase
    # timed alone (the attraction on the main stream instead of overlapped)
    t.set_Y(y_s)
    t.set_state(v_s, None, 0)
    t.set_profiling(True, serial=True)
    t.get_profile()
    protocol(t, W, K, theta, lr)
    sprof, siters = t.get_profile()
    t.set_profiling(False)
    sphase = {k: v / max(siters, 1) for k, v in sprof.items()}
    dominant = max(sphase, key=sphase.get)  # from the serial replay: each phase timed alone
    from paper_2401_13708_gb300 import measure_peaks
    mpeaks = measure_peaks(local)
    hbm = peaks.get("hbm_gbs")
    fp64_rec = fp64_ops_record()
    kernels = {}
    for ph, bpp in BYTES_PER_POINT.items():
        gbs = bpp * n / (sphase[ph] * 1e-3) / 1e9
        kernels[ph] = {"bound": "hbm", "ms": sphase[ph], "algorithmic_bytes": bpp * n, "achieved": gbs,
                       "unit": "GB/s", "peak": hbm, "frac": gbs / hbm if hbm else None}
        if ph in fp64_rec and mpeaks["fp64_fma_tflops"]:
            # float64-pipe-bound phases: their FP64 rate against the measured FP64 FMA peak
            tf = fp64_rec[ph] * n / (sphase[ph] * 1e-3) / 1e12
            kernels[ph]["bound"] = "fp64"
            kernels[ph]["fp64"] = {"flop_per_point": fp64_rec[ph], "achieved": tf, "unit": "TFLOP/s",
                                   "peak": mpeaks["fp64_fma_tflops"], "frac": tf / mpeaks["fp64_fma_tflops"],
                                   "peak_basis": "hts_measure_peaks float64 FMA, this run"}
    abytes = ATTRACT_BYTES_PER_NNZ * int(w.nnz) + ATTRACT_BYTES_PER_ROW * n
    agbs = abytes / (sphase["attract"] * 1e-3) / 1e9
    kernels["attract"] = {"bound": "hbm", "ms": sphase["attract"], "algorithmic_bytes": abytes, "achieved": agbs,
                          "unit": "GB/s", "peak": hbm, "frac": agbs / hbm if hbm else None,
                          "note": "runs overlapped with the walk in the timed iteration"}
    wflop = flops / (sphase["walk"] * 1e-3) / 1e12
    # special-function unit: rsqrt, log2 and reciprocal per interaction (3 ops)
    mufu_tops = 3.0 * (acc + pairs) / K / (sphase["walk"] * 1e-3) / 1e12
    mufu_peak = props.multi_processor_count * 16 * sm_mhz * 1e6 / 1e12
    kernels["walk"] = {"bound": "alu", "ms": sphase["walk"], "achieved": wflop, "unit": "TFLOP/s",
                       "peak": fp32_peak, "frac": wflop / fp32_peak,
                       "frac_of_measured_fp32": wflop / mpeaks["fp32_fma_tflops"]
                       if mpeaks["fp32_fma_tflops"] else None,
                       "mufu": {"achieved_tops": mufu_tops, "peak_tops": mufu_peak, "frac": mufu_tops / mufu_peak,
                                "peak_basis": "SMs x 16 x sampled SM clock; measured: %.2f Tops/s" %
                                              mpeaks["mufu_rsqrt_tops"]}}

    # ---- end to end through the C ABI, all iteration state in host memory -
    k_e2e = K  # the same iterations as the device-timed segment
    yh = torch.from_numpy(np.ascontiguousarray(y_s)).pin_memory()
    t.set_Y(y_s)                                   # the segment's start state (velocity restored)
    t.set_state(v_s, None, 0)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for k in range(k_e2e):
        t.update_Y(yh)                             # this step's input: Y from pinned host memory
        protocol(t, W + k, 1, theta, lr)
        t.get_Y(yh)                                # this step's result: Y back to the host
    torch.cuda.synchronize()
    barrier(world)
    dt = max_over_ranks(time.perf_counter() - t0, world)
    e2e = {"value": k_e2e * world / dt, "unit": UNIT, "steps": k_e2e,
           "h2d_bytes_per_step": int(yh.numel() * 8), "d2h_bytes_per_step": int(yh.numel() * 8),
           "call": "per step: hts_update_Y (pinned host Y in; the optimiser state stays in the context) -> "
                   "hts_step(1) -> hts_get_Y (pinned host Y out); the same iterations as the timed segment, "
                   "from the same state"}
    t.close()

    # ---- FP64 GPU path on the same segment --------------------------------
    t64 = HyperbolicTSNE(precision="fp64", device=local)
    t64.set_P(w.indptr, w.indices, w.values)
    t64.set_Y(y_s)
    t64.set_state(v_s, None, 0)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    protocol(t64, W, k64, theta, lr)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = max_over_ranks(e0.elapsed_time(e1), world)
    value64 = k64 * world / (ms64 / 1e3)
    t64.close()

    # ---- oracle: error gate and CPU baseline (rank 0 only) ---------------
    errs, cpu = {}, None
    if rank == 0 and not args.no_oracle:
        rng = np.random.default_rng(args.seed + 2)
        rows = np.sort(rng.choice(n, size=min(args.sample_rows, n), replace=False))
        for name, ys in gate_states.items():
            ref, t_or, cores = oracle_pass(w, ys, theta, rows)
            g, z = g32[name]
            errs[name] = {"grad_rel_err": float(np.linalg.norm(g[rows] - ref["g"]) / np.linalg.norm(ref["g"])),
                          "worst_row_err": worst_row_err(g[rows], ref),
                          "z_rel_err": float(abs(z - ref["Z"]) / ref["Z"])}
            if name == "y0":
                cpu = {"value": 1.0 / t_or, "unit": UNIT, "cores": cores, "kind": "oracle",
                       "cpu_model": cpu_model(),
                       "sample": (f"one FP64 oracle pass at N={n} on Y0: literal-insertion tree, BH walks of all "
                                  f"{n} points (for Z) and gradient rows for {len(rows)} sampled points; "
                                  f"{t_or:.1f} s")}
        # one thread: the tree once and a bounded sample of row walks, extrapolated
        import oracle
        all_cores = oracle.set_threads(0)
        oracle.set_threads(1)
        t0 = time.time()
        tree = oracle.PreparedTree(y0)
        t_tree = time.time() - t0
        srows = rng.choice(n, size=min(4000, n), replace=False)
        t0 = time.time()
        tree.walk_rows(srows, w.indptr, w.indices, np.asarray(w.values, dtype=np.float64), theta, 1.0, 1.0)
        t_rows = time.time() - t0
        tree.close()
        oracle.set_threads(all_cores)
        t1 = t_tree + t_rows * n / len(srows)
        if cpu is not None:
            cpu["single_thread"] = {"value": 1.0 / t1, "unit": UNIT, "cores": 1,
                                    "sample": (f"tree built once ({t_tree:.2f} s) + {len(srows)} row walks "
                                               f"({t_rows:.2f} s) at Y0, extrapolated to {n} rows")}

    if rank != 0:
        return
    r_end = np.linalg.norm(y_end, axis=1)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(n, theta), "n": n,
                   "nnz": int(w.nnz), "theta": theta, "precision": "fp32_mixed",
                   "protocol": f"iterations {W}..{W + K - 1} of 250 (exaggeration 12, momentum 0.5) + 750 "
                               f"(1, 0.8), lr = N/12000, Y0 ~ N(0, 1e-4 I)",
                   "l2": "inputs larger than L2 (CSR ~%.2f GB)" % (w.nnz * 8 / 1e9),
                   "parallelism": f"replicas x{world}", "generate_s": round(t_gen, 1),
                   "launch_shapes": {"walk_threads_per_block": walk_block, "attract_lanes_per_row": attract_lanes,
                                     "chosen_by": "--shapes" if args.shapes else "hts_autotune after the warm-up"}},
        "kernel_rooflines": {"source": "the timed segment replayed with each phase timed alone (CUDA events)",
                             "hbm_peak_basis": "MEASURED_PEAKS.json hbm_gbs (copy, read + write)",
                             "phase_ms_per_step": sphase, "kernels": kernels},
        "measured_peaks": dict(mpeaks, note="this library's microbenchmarks (hts_measure_peaks), this run"),
        "phase_ms_per_step": {k: v / max(piters, 1) for k, v in prof.items()},
        "walk_counters_per_step": {"accepted_cells": acc / K, "leaf_pairs": pairs / K,
                                   "warp_node_visits": visits / K, "criterion_tests": crit / K,
                                   "interactions_per_point": (acc + pairs) / max(queries, 1),
                                   "replay_reproduced_trajectory": replay_same},
        "y_end": {"max_radius": float(r_end.max()), "boundary_stop_would_fire": bool(np.any(r_end > 1 - 1e-4))},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": {"kernel": "walk_f32_kernel (BH tree walk)", "bound": "alu", "achieved": achieved,
                     "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": traffic,
                     "frac_of_measured_fp32": achieved / mpeaks["fp32_fma_tflops"]
                     if mpeaks["fp32_fma_tflops"] else None,
                     "dominant_phase": dominant, "walk_ms": walk_ms,
                     "peak_basis": "FP32 lanes: %d SMs x 128 x 2 flop x %.0f MHz (sampled SM clock)" % (
                         props.multi_processor_count, sm_mhz)},
        # last, so that they stay in view when only the end of the line is kept
        "fp64_gpu": {"value": value64, "unit": UNIT, "fp32_mixed_speedup": ms64 / ms32_seg, "steps": k64,
                     "ms_per_step": ms64 / k64, "fp32_mixed_ms_per_step_same_segment": ms32_seg / k64},
        "grad_error_gate": errs,
        "grad_rel_err": max((e["grad_rel_err"] for e in errs.values()), default=None),
        "grad_worst_row_err": max((e["worst_row_err"] for e in errs.values()), default=None),
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# per-configuration report (--suite): all five workloads, fixed iteration counts
# ---------------------------------------------------------------------------

def run_suite(args, rank, world, local):
    """One JSON line per (workload, path): iterations/s and wall time to the
    workload's fixed iteration count on one GPU (CUDA events around the
    hts_step calls, after 3 warm-up iterations from the same start), and the
    oracle's time per iteration on this host's cores.  FP64 runs longer than
    ~30 s are timed on a prefix of the schedule and extrapolated (labelled)."""
    if rank != 0:
        return
    import torch

    import oracle
    from paper_2401_13708_gb300 import HyperbolicTSNE, inputs
    cores = oracle.set_threads(0)
    model = cpu_model()
    dev = f"cuda:{local}"

    def schedule(n_total, ee, exag, mom1, mom2, lr):
        return [(ee, exag, lr, mom1), (n_total - ee, 1.0, lr, mom2)]

    def gpu_time(prec, w, y0, sched, theta, max_iters=None, segments=None, lr_scale=None, graphs=False,
                 split_rule="equal_length"):
        t = HyperbolicTSNE(precision=prec, device=local, split_rule=split_rule)
        t.set_P(w.indptr, w.indices, w.values)
        t.set_Y(y0)
        if segments is not None:
            t.set_segments(segments, lr_scale)
        shapes = t.autotune(theta, 2) if theta > 0 else None
        t.set_graphs(graphs)
        t.step(3, theta, sched[0][1], sched[0][2], sched[0][3])  # warm-up (and capture), then restart
        t.set_Y(y0)
        total = sum(s[0] for s in sched)
        run = total if max_iters is None else min(total, max_iters)
        left, todo = run, []
        for k, ex, lr, mom in sched:
            m = min(k, left)
            if m > 0:
                todo.append((m, ex, lr, mom))
            left -= m
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for m, ex, lr, mom in todo:
            t.step(m, theta, ex, lr, mom)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        t.close()
        out = {"iters_per_s": run / (ms / 1e3), "timed_iters": run, "schedule_iters": total,
               "wall_s_to_schedule": ms / 1e3 * total / run, "extrapolated": run < total}
        if shapes:
            out["launch_shapes"] = list(shapes)
        return out

    def emit(line):
        line.update({"data": "synthetic", "n_gpus": 1, "unit": "iters/s"})
        print(json.dumps(line), flush=True)

    def oracle_iters(w, y0, k, theta, exag, lr, mom, nseg_slices=None):
        t0 = time.time()
        if nseg_slices is None:
            oracle.step(y0, np.zeros_like(y0), w.indptr, w.indices, w.values, k, theta, exag, lr, mom)
        else:
            for (a, b, ip, ix, vv, lr_s) in nseg_slices:
                oracle.step(y0[a:b], np.zeros_like(y0[a:b]), ip, ix, vv, k, theta, exag, lr_s, mom)
        dt = (time.time() - t0) / k
        return {"s_per_iter": dt, "iters_per_s": 1.0 / dt, "iters_timed": k, "cores": cores, "cpu_model": model}

    want = {v.strip() for v in args.workloads.split(",") if v.strip()}

    # Gaussian mixture, N = 2000, FP64 CSR; 100 iterations, exaggeration 12 for 25, lr 1, momentum 0.5
    w = inputs.make_workload("gaussian_mixture", seed=args.seed, device=dev)
    sched = schedule(100, 25, 12.0, 0.5, 0.5, 1.0)
    for theta in ((0.0, 0.5) if "gaussian_mixture" in want else ()):
        line = {"workload": inputs.WORKLOADS["gaussian_mixture"], "n": w.n, "nnz": w.nnz, "theta": theta,
                "iterations": 100, "schedule": "25 x (exaggeration 12) + 75 x 1, lr 1, momentum 0.5"}
        line["fp64_gpu"] = gpu_time("fp64", w, w.y0, sched, theta, graphs=True)
        line["fp32_mixed_gpu"] = gpu_time("fp32", w, w.y0, sched, theta, graphs=True)
        line["fp32_mixed_gpu_eager"] = gpu_time("fp32", w, w.y0, sched, theta)
        line["oracle"] = oracle_iters(w, w.y0, 100, theta, 12.0, 1.0, 0.5)
        emit(line)

    # MNIST-shaped, binary-tree and single-cell-like: the paper's protocol, 1000 iterations, lr = N / 12000
    for name, thetas in (("mnist_like", (0.5,)), ("binary_tree", (0.2, 0.5, 0.8)), ("single_cell", (0.5, 0.8))):
        if name not in want:
            continue
        w = inputs.make_workload(name, seed=args.seed, device=dev)
        lr = w.n / 12000.0
        sched = schedule(1000, 250, 12.0, 0.5, 0.8, lr)
        for theta in thetas:
            line = {"workload": inputs.WORKLOADS[name], "n": w.n, "nnz": w.nnz, "theta": theta,
                    "iterations": 1000,
                    "schedule": "250 x (exaggeration 12, momentum 0.5) + 750 x (1, 0.8), lr = N/12000"}
            if args.split_rule != "equal_area":
                line["fp32_mixed_gpu"] = gpu_time("fp32", w, w.y0, sched, theta)
            if theta == 0.5 and args.split_rule != "equal_length":
                # Sec. 5.2.2 (Time Gain by Splitting Choices): the same run on equal-area splits
                line["fp32_mixed_gpu_equal_area"] = gpu_time("fp32", w, w.y0, sched, theta, split_rule="equal_area")
                if "fp32_mixed_gpu" in line:
                    t_len = 1.0 / line["fp32_mixed_gpu"]["iters_per_s"]
                    t_area = 1.0 / line["fp32_mixed_gpu_equal_area"]["iters_per_s"]
                    line["equal_length_time_gain"] = {"per_iteration": 1.0 - t_len / t_area,
                                                      "note": "1 - t(equal length) / t(equal area), FP32-mixed"}
            if args.split_rule == "equal_area":
                emit(line)
                continue
            f64 = gpu_time("fp64", w, w.y0, sched, theta, max_iters=60 if name == "single_cell" else 250)
            line["fp64_gpu"] = f64
            f32p = gpu_time("fp32", w, w.y0, sched, theta, max_iters=f64["timed_iters"])
            line["fp32_mixed_speedup_over_fp64"] = {"iters": f64["timed_iters"],
                                                    "speedup": f32p["iters_per_s"] / f64["iters_per_s"]}
            if theta == 0.5:
                k = 1 if name == "single_cell" else 10
                line["oracle"] = oracle_iters(w, w.y0, k, theta, 12.0, lr, 0.5)
            emit(line)

    # 64 mixtures in one context, 500 iterations (125 exaggerated), lr = n_s / 12000
    if "batched_mixtures" not in want:
        return
    w = inputs.make_batched(64, seed=args.seed, device=dev)
    off = w.extra["offsets"]
    sizes = np.diff(off).astype(np.float64)
    sched = schedule(500, 125, 12.0, 0.5, 0.8, 1.0)
    line = {"workload": "64 batched mixtures N~logU(500,20000), D=50, 3-20 components, perplexity {10,30,50}",
            "n": w.n, "nnz": w.nnz, "theta": 0.5, "iterations": 500,
            "schedule": "125 x (exaggeration 12, momentum 0.5) + 375 x (1, 0.8), lr = n_s/12000 per embedding"}
    line["fp32_mixed_gpu_graphs"] = gpu_time("fp32", w, w.y0, sched, 0.5, segments=off, lr_scale=sizes / 12000.0,
                                             graphs=True)
    line["fp32_mixed_gpu_eager"] = gpu_time("fp32", w, w.y0, sched, 0.5, segments=off, lr_scale=sizes / 12000.0)
    slices = []
    for sg in range(len(off) - 1):
        a, b = int(off[sg]), int(off[sg + 1])
        e0, e1 = int(w.indptr[a]), int(w.indptr[b])
        slices.append((a, b, (w.indptr[a:b + 1] - e0).astype(np.int64), (w.indices[e0:e1] - a).astype(np.int32),
                       np.asarray(w.values[e0:e1], dtype=np.float64), sizes[sg] / 12000.0))
    line["oracle"] = oracle_iters(w, w.y0, 1, 0.5, 12.0, None, 0.5, nseg_slices=slices)
    emit(line)


def main():
    args = parse()
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.suite:
        run_suite(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
