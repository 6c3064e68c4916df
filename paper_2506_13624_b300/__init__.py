"""B300-native branch-MPC solver (multiple-shooting AL-iLQR over scenario trees).

The compute path is the CUDA library ``libbmpc.so`` behind the C ABI of
``include/bmpc.h``; :mod:`paper_2506_13624_b300.bmpc` is its ctypes binding.
"""
from .bmpc import Batch, Opts, default_opts, lib, solve, status_str  # noqa: F401

__all__ = ["Batch", "Opts", "default_opts", "lib", "solve", "status_str"]
