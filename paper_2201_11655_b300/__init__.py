"""B300-native per-vertex directed 3/4-motif counting (VDMC, arXiv 2201.11655).

The counting runs in the CUDA library ``libvdmc.so`` behind a C ABI
(``include/vdmc.h``); :mod:`paper_2201_11655_b300.vdmc` is its thin Python
binding.  Importing this package does not load the library; the binding
loads it on first use and raises if it is missing.
"""
__all__ = ["vdmc", "synth"]
