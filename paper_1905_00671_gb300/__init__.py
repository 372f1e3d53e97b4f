"""GB300-native stabilized implicit u-p material point method (Zhao & Choo).

The compute path is the CUDA library built from csrc/ behind the C-ABI declared
in include/mpm.h; `paper_1905_00671_gb300.mpm` is its thin ctypes binding.
Importing this package loads nothing; the binding loads the library on first
use and raises if it is missing.
"""
__all__ = ["inputs", "mpm"]
