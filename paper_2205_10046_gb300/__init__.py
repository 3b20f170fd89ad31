"""GB300-native NEP3 energy/force/virial evaluation and NVE dynamics (arXiv:2205.10046).

Submodules:
  nep        ctypes binding of libnep (include/nep.h); the CUDA kernels do all the work
  workloads  seeded synthetic structures, random model weights and velocities
  build      nvcc build of libnep.so (sm_103a)
"""
