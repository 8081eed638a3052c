"""GB300-native approximate Gauss-Newton gain calibration (arxiv 2412.10072).

Submodules are imported lazily: ``synth`` (seeded synthetic observations),
``qc`` (binding of libqc.so, the CUDA solver behind the C ABI of
include/qc.h) and ``build`` (nvcc build of libqc.so).
"""
__all__ = ["build", "qc", "synth"]
