"""GB300-native NGS-FAS solver for the Richards equation.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/richards.h``); ``paper_2606_04292_gb300.richards`` is its ctypes
binding and :mod:`.workloads` generates seeded synthetic problems.
"""
from . import workloads  # noqa: F401
