"""GB300 (sm_103a) library for the tensorized approximation (TA) of the long-range
two-electron integrals tensor (Badreddine, Chollet, Grigori, arXiv 2210.13069).

Submodules:
  build_lib -- compiles csrc/*.cu into _build/liblrtei.so (nvcc, sm_103a)
  lrtei     -- thin ctypes binding of the C ABI in include/lrtei.h
  synth     -- seeded synthetic molecules and densities (inputs only)

Nothing is imported eagerly: importing the package does not load the CUDA library.
"""

__all__ = ["build_lib", "lrtei", "synth"]
