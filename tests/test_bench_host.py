"""Host logic of bench.py that needs no GPU: the paper's iteration schedule,
the per-row error measure of the gradient gate, and the rule that a committed
per-point float64 count is used only while its kernel source is unchanged."""
import json
import os
import shutil

import numpy as np

import bench


class _Recorder:
    def __init__(self):
        self.calls = []

    def step(self, n, theta, exag, lr, mom):
        self.calls.append((n, theta, exag, lr, mom))


def test_protocol_schedule_sec_5_1():
    # 250 iterations with exaggeration 12 and momentum 0.5, then 1 and 0.8
    cases = {
        (0, 5): [(5, 12.0, 0.5)],
        (5, 995): [(245, 12.0, 0.5), (750, 1.0, 0.8)],
        (248, 5): [(2, 12.0, 0.5), (3, 1.0, 0.8)],
        (250, 10): [(10, 1.0, 0.8)],
        (600, 3): [(3, 1.0, 0.8)],
    }
    for (it0, k), want in cases.items():
        t = _Recorder()
        bench.protocol(t, it0, k, 0.5, 83.3)
        assert [(n, e, m) for n, _, e, _, m in t.calls] == want
        assert all(th == 0.5 and lr == 83.3 for _, th, _, lr, _ in t.calls)
        assert sum(c[0] for c in t.calls) == k


def test_worst_row_error_is_relative_to_the_force_terms():
    # two rows; the reference force terms give each row its own scale
    ref = {"g": np.array([[1.0, 0.0], [0.0, 0.0]]),
           "fattr": np.array([[0.25, 0.0], [1.0, 0.0]]),
           "frep": np.array([[0.0, 0.0], [2.0, 0.0]]), "Z": 2.0}
    g = np.array([[1.1, 0.0], [0.0, 0.4]])
    # row 0: |d| = 0.1, scale max(4 (0.25 + 0), |g| = 1) = 1 -> 0.1
    # row 1: |d| = 0.4, scale 4 (1 + 2 / 2) = 8 -> 0.05
    assert abs(bench.worst_row_err(g, ref) - 0.1) < 1e-15
    assert bench.worst_row_err(ref["g"], ref) == 0.0


def test_fp64_counts_follow_their_sources(tmp_path, monkeypatch):
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "fp64_ops_step_n200k.txt")))
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, "profiles", "fp64_ops_step_n200k.txt"), root / "profiles")
    shutil.copytree(os.path.join(bench.ROOT, "paper_2401_13708_gb300", "csrc"),
                    root / "paper_2401_13708_gb300" / "csrc")
    monkeypatch.setattr(bench, "ROOT", str(root))
    same = bench.fp64_ops_record()
    # a phase is rated only if its source hashes as recorded
    csrc = root / "paper_2401_13708_gb300" / "csrc"
    import hashlib
    for ph, f in rec["phase_source"].items():
        ok = hashlib.sha256((csrc / f).read_bytes()).hexdigest() == rec["sources_sha256"][f]
        assert (ph in same) == ok
        if ok:
            assert same[ph] == rec["fp64_flop_per_point"][ph]
    # an edited source drops its phase and keeps the others
    src = csrc / rec["phase_source"]["update"]
    src.write_bytes(src.read_bytes() + b"\n// edited\n")
    after = bench.fp64_ops_record()
    assert "update" not in after
    assert {k: v for k, v in same.items() if k != "update"} == after
