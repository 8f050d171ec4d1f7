"""GB300-native crossbar nodal solver (the hot path of XbarSim, arXiv 2410.19993).

Submodules:
  inputs    seeded synthetic workloads (no solver arithmetic)
  xbar      ctypes binding of the CUDA library libxbar.so (C ABI in include/xbar.h)
  build     nvcc build of libxbar.so for sm_103a

The binding is imported lazily so that ``inputs`` can be used on machines
without the compiled library; every compute call goes through libxbar.so and
fails loudly when it is missing.
"""
__all__ = ["inputs", "xbar", "build"]
