"""GB300-native (sm_103a) ETD2 + embedded-boundary + level-set path of
Liu & Liu, arXiv 2209.15095.

  csrc/      CUDA kernels and the C-ABI library (libetd_gb300.so)
  build.py   compiles the library with nvcc for sm_103a
  etd.py     thin ctypes binding over the C-ABI (argument marshalling only)
  inputs.py  seeded synthetic initial data for the workloads

The binding is imported lazily so that the input generators can be read on
a machine without a GPU.
"""

__all__ = ["etd", "inputs", "build"]
