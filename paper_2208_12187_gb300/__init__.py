"""GB300-native trust-region-reflective curve fitting (libgbfit).

The compute path is the CUDA library built from ``csrc/`` for sm_103a; the
Python layer (``gbfit``) only marshals arguments through its C ABI.
``synth`` draws seeded synthetic problems shaped like the paper's workloads.
"""
from . import build, gbfit, synth  # noqa: F401

__all__ = ["build", "gbfit", "synth"]
