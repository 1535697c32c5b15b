"""The C ABI library loads on a CPU-only host and exports every entry point
declared in include/hts.h (no compute calls: there is no GPU here)."""
import ctypes
import os
import re

import pytest

from paper_2401_13708_gb300 import _lib, buildlib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "hts.h")).read()
    return sorted(set(re.findall(r"^HTS_API[^;(]*?\b(hts_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["hts_create", "hts_destroy", "hts_set_P", "hts_set_Y", "hts_step", "hts_get_Y", "hts_grad",
                     "hts_kl", "hts_last_error"]:
        assert required in names
    assert sorted(_lib.EXPORTS) == names


def test_library_builds_and_exports_every_declared_symbol():
    path = buildlib.build()
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_null_and_invalid_arguments_are_rejected_without_a_gpu():
    lib = _lib.load()
    assert lib.hts_create(None, None) == -1
    assert lib.hts_last_error(None) == b"no context"
    cfg = _lib.HtsConfig()
    lib.hts_default_config(ctypes.byref(cfg))
    assert cfg.precision == _lib.FP32_MIXED and cfg.eps == pytest.approx(1e-5) and cfg.metric_pow == 1
    cfg.precision = 7
    ctx = ctypes.c_void_p()
    assert lib.hts_create(ctypes.byref(ctx), ctypes.byref(cfg)) == -1
    assert lib.hts_step(None, 1, 0.5, 1.0, 1.0, 0.5) == -1


def test_error_codes_match_the_header():
    text = open(os.path.join(ROOT, "include", "hts.h")).read()
    codes = {int(v): k for k, v in re.findall(r"^#define (HTS_E\w+) \((-\d+)\)", text, flags=re.M)}
    assert codes == _lib.ERRORS
    assert re.search(r"^#define HTS_OK 0", text, flags=re.M)
