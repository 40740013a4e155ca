"""GB300-native multiscale, symmetric, debiased Sinkhorn (Feydy et al., MICCAI 2019).

``otgb`` is the ctypes binding of the CUDA library libotgb.so (C ABI in
include/otgb.h); ``synth`` draws the seeded synthetic inputs; ``build`` compiles
the library for sm_103a; ``replicas`` combines the timings of independent
replicas run one per GPU.  Importing the package does not load the library:
the first call through ``otgb`` does, and fails loudly when it is missing.
"""
__all__ = ["build", "otgb", "replicas", "synth"]
