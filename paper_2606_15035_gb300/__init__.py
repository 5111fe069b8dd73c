"""GB300 (sm_103a) implementation of the energy-conserving unstaggered potential PIC step.

The compute path is the CUDA library built from ``csrc/`` (C-ABI in include/pic.h);
``sim`` is its Python binding.  Importing this package does not load the library; the
first binding call does, and raises if it has not been built.
"""

from . import build, sim  # noqa: F401

__all__ = ["build", "sim"]
