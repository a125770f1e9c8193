"""GB300-native Vlasov-Hybrid (VHS) time step: push, VHS reconstruction,
velocity moment and spectral Poisson solve in hand-written sm_103a CUDA,
behind the C ABI of include/avl.h.

``from paper_1804_03901_gb300 import avl`` loads the compiled library and
raises if it is missing (build it with ``paper_1804_03901_gb300.build.build()``).
"""
