"""GB300-native (sm_103a) CV-ADAPT-VQE hot path (arXiv 2606.05297).

Layers: libcvq.so (CUDA kernels + C ABI, include/cvq.h) <- cvq (ctypes
binding) <- adapt (BFGS + ADAPT driver, Lanczos).  workloads holds the seeded
synthetic inputs.
"""
