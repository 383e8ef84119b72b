"""GB300 (sm_103a) prover for zkVC's CRPC + PSQ matrix-multiplication circuit under
Groth16 over BN254 (arXiv 2504.12217).

``native``  ctypes binding of libzkvc.so (the C ABI of include/zkvc.h)
``build``   in-tree nvcc build of libzkvc.so
``inputs``  seeded synthetic workloads (random draws only)
"""
