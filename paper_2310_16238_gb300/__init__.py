"""GB300-native regularized stratified / time-varying Cox fitting (arXiv 2310.16238).

The compute path is a C-ABI shared library of hand-written sm_103a CUDA kernels
(``csrc/``, declared in ``include/cox.h``); ``paper_2310_16238_gb300.cox`` is a thin ctypes
binding to it. ``synth`` draws seeded synthetic inputs. Importing this package does not load
the CUDA library; the first call into ``cox`` does, and raises if it is missing.
"""
__all__ = ["cox", "synth"]
