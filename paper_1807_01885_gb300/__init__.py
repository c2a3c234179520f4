"""GB300-native FFT-BEM for non-adhesive and adhesive contact with a coated half-space.

The compute path lives in ``libbem.so`` (hand-written sm_103a CUDA behind the C ABI
declared in ``include/bem.h``); ``paper_1807_01885_gb300.bem`` is a thin ctypes
binding with the same entry-point names.  ``inputs`` holds the seeded synthetic
input generators (height maps, rough surfaces, layer parameters).

Importing this package does not load the library; the first call into ``bem``
does, and raises if the CUDA library is missing (there is no CPU fallback).
"""
__all__ = ["bem", "inputs"]
