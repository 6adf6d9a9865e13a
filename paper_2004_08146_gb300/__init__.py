"""GB300-native GD-lambda-AMG hot path (Hermitian Wilson-clover eigensolver).

The compute path lives in ``libqcd.so`` (hand-written sm_103a CUDA behind a C
ABI, see ``include/qcd.h``); ``paper_2004_08146_gb300.qcd`` is the thin ctypes
binding.  Importing this package does not load the library: ``qcd`` raises
when ``libqcd.so`` is missing, there is no fallback.
"""
__all__ = ["qcd", "synth", "workloads", "autograd"]
