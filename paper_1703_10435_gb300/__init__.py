"""GB300 (sm_103a) pipeline for the local problems of the Multiscale
Hybrid-Mixed method: batched assembly, zero-mean Neumann factorisation,
multi-RHS solves and face-integral reduction into the skeleton system.

Submodules:
  build      compiles libmhm.so (nvcc, sm_103a) in-tree
  mhm        ctypes binding of include/mhm.h, same function names
  pipeline   device-buffer management around the C calls
  workloads  seeded synthetic inputs (no method arithmetic)
"""
