"""GB300-native KPM observable engine for the RMFT vortex solver of arXiv:2212.05685.

The compute path lives in the CUDA library `libkpm.so` built from `csrc/` for
sm_103a; `kpm.py` is a thin ctypes binding with the same entry-point names as
the C ABI in `include/kpm.h`.  Importing this package loads nothing: call
`paper_2212_05685_gb300.kpm.load()` (done lazily by every binding function).
"""
__all__ = ["inputs", "kpm"]
