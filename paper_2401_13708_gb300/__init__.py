"""GB300-native hyperbolic t-SNE gradient ("Accelerating hyperbolic t-SNE", arXiv 2401.13708).

The computation lives in the CUDA library libhts (csrc/, C ABI in
include/hts.h); `HyperbolicTSNE` is its Python binding.  `inputs` holds the
seeded synthetic workloads.  Importing the package does not load the
library; constructing a HyperbolicTSNE does, and raises if it is missing.
"""
from .api import (EQUAL_AREA, EQUAL_LENGTH, EXACT_KL, FP32_MIXED, FP64, PAPER_EQ, HtsError,  # noqa: F401
                  HyperbolicTSNE, measure_peaks)


def build(force: bool = False) -> str:
    """Compile libhts.so for sm_103a (in-tree) and return its path."""
    from . import buildlib
    return buildlib.build(force=force)
