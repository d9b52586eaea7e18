"""GB300-native partial-wave-analysis likelihood (Berger, arXiv:1108.5882, Sec. 2).

The compute path is libpwa.so (hand-written CUDA for sm_103a behind the C ABI of
include/pwa.h); ``pwa`` is its thin ctypes binding, ``inputs`` the seeded synthetic inputs.
Submodules are imported lazily so that ``inputs`` can be used without torch or a GPU.
"""
__all__ = ["pwa", "inputs", "build"]
